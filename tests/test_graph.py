"""The random-frequency mode-locked graph (Sec. II.C "Quenched random frequencies", "Graph generation",
Eq. (gamma_scaling)): the oracle's brute-force generator is pinned by the comb it must reproduce for
equally spaced frequencies and by the connectivity the paper's linewidth is chosen to match; the
library's generator (a different algorithm) must give the identical list; the oracle's PT engine runs
on such graphs with the constraint kept and the running energy exact."""
import numpy as np
import pytest

import oracle
import paper_2511_13508_gb300 as pkg
from paper_2511_13508_gb300 import workload


@pytest.mark.parametrize("N", [4, 6, 9, 16, 25, 40])
def test_equally_spaced_frequencies_give_the_comb(N):
    w = np.arange(N) / (N - 1)
    assert np.array_equal(oracle.fmc_graph(w), oracle.enumerate_quads(N)[: len(oracle.fmc_graph(w))])
    assert len(oracle.fmc_graph(w)) == len(oracle.enumerate_quads(N))


@pytest.mark.parametrize("N", [32, 64])
def test_linewidth_keeps_the_comb_connectivity(N):
    """gamma = 1/(2(N-1)) is chosen so that random frequencies give as many interactions as the comb."""
    rng = np.random.default_rng(N)
    cnt = [len(oracle.fmc_graph(workload.random_frequencies(N, int(s)))) for s in rng.integers(0, 10 ** 6, 16)]
    comb = len(oracle.enumerate_quads(N))
    assert abs(np.mean(cnt) / comb - 1.0) < 0.05, (np.mean(cnt), comb)


def test_every_listed_interaction_matches_and_splittings_vary():
    w = workload.random_frequencies(24, 7)
    g = oracle.fmc_graph(w)
    gamma = 1.0 / (2 * 23)
    lhs = w[g[:, 0]] + w[g[:, 3]] - w[g[:, 1]] - w[g[:, 2]]
    assert np.all(np.abs(lhs) < gamma)
    assert len({tuple(sorted(q)) for q in g.tolist()}) <= len(g)
    many = np.concatenate([oracle.fmc_graph(workload.random_frequencies(24, s)) for s in range(8)])
    assert np.any(np.any(np.diff(many, axis=1) < 0, axis=1))  # splittings other than {a,d}|{b,c} occur


@pytest.mark.parametrize("N", [8, 16, 32, 64])
def test_library_generator_matches_the_oracle(N):
    pkg.build()
    for seed in range(3):
        w = workload.random_frequencies(N, 100 * N + seed)
        assert np.array_equal(pkg.fmc_graph(w), oracle.fmc_graph(w))
    assert np.array_equal(pkg.fmc_graph(np.arange(N) / (N - 1)), pkg.enumerate_quads(N))


def test_library_generator_rejects_bad_input():
    pkg.build()
    with pytest.raises(pkg.PTError):
        pkg.fmc_graph(np.array([0.1, 0.3, 0.2, 0.5, 0.9]))  # not ascending
    with pytest.raises(pkg.PTError):
        pkg.fmc_graph(np.linspace(0, 1, 8), gamma=0.0)


def _rand_state(N, rng):
    g = rng.standard_normal(N)
    u = np.sqrt(N) * np.abs(g) / np.linalg.norm(g)
    return np.sqrt(u) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))


def test_energy_on_a_random_graph_keeps_the_global_phase_but_not_the_comb_gauge():
    N = 16
    w = workload.random_frequencies(N, 3)
    g = oracle.fmc_graph(w)
    J = workload.couplings(N, len(g), 4)
    rng = np.random.default_rng(5)
    a = _rand_state(N, rng)
    E = oracle.energy(N, g, J, a)
    assert abs(oracle.energy(N, g, J, a * np.exp(0.7j)) - E) < 1e-12
    Eg = oracle.energy(N, g, J, a * np.exp(1j * 0.9 * np.arange(N)))
    assert abs(Eg - E) > 1e-3  # the comb gauge is a symmetry of the comb only
    # a pair move: Delta H against full recomputation
    j, k = 3, 11
    aj, ak = 0.8 * np.exp(0.2j), 1.1 * np.exp(-1.3j)
    b = a.copy(); b[j], b[k] = aj, ak
    assert abs(oracle.delta_h(N, g, J, a, j, k, aj, ak) - (oracle.energy(N, g, J, b) - E)) < 1e-11


def test_oracle_pt_on_random_graphs():
    Ns = [16, 24]
    graphs = [oracle.fmc_graph(workload.random_frequencies(n, 10 + n)) for n in Ns]
    Js = [workload.couplings(n, len(g), 20 + n) for n, g in zip(Ns, graphs)]
    pt = oracle.OraclePT(Ns, Js, workload.geometric_ladder(0.4, 1.6, 4), 2, 9, swap_every=8, measure_every=4,
                         resync_every=0, graphs=graphs)
    pt.sweep(256)
    a, E = pt.state()
    off = 0
    for s, n in enumerate(Ns):
        for c in range(2 * 4):
            x = a[off: off + n]
            assert abs((np.abs(x) ** 4).sum() - n) < 1e-10 * n
            assert abs(oracle.energy(n, graphs[s], Js[s], x) - E[s * 8 + c]) < 1e-9
            off += n


@pytest.mark.parametrize("N,z", [(64, 4), (512, 8), (2048, 16)])
def test_sparse_comb_graph(N, z):
    """Finite connectivity: round(z N / 4) distinct comb quadruplets, z per mode on average."""
    g = workload.sparse_comb_graph(N, z, 3)
    assert len(g) == round(z * N / 4)
    assert np.all(g[:, 0] + g[:, 3] == g[:, 1] + g[:, 2])
    assert np.all((g[:, 0] < g[:, 1]) & (g[:, 1] < g[:, 2]) & (g[:, 2] < g[:, 3])) and g.min() >= 0 and g.max() < N
    assert len({tuple(q) for q in g.tolist()}) == len(g)
    assert abs(np.bincount(g.ravel(), minlength=N).mean() - z) < 1e-12
    if N == 64:  # every listed quadruplet belongs to the comb list
        comb = {tuple(q) for q in oracle.enumerate_quads(N).tolist()}
        assert all(tuple(q) in comb for q in g.tolist())


@pytest.mark.parametrize("kind", ["random", "comb", "sparse"])
def test_incidence_records_decode_to_the_oracle_fields(kind):
    """The FP32 quadruplet-list kernels read one record per (mode, quadruplet holding it): three row offsets
    A, B, C and the positions of the four factors, so that the term is J a_A a_B conj(a_C).  Decoded on the
    host, every record must give the oracle's contribution of its quadruplet to the local field of its mode
    (Sec. III.A.3), the positions must name where each mode sits, and the records of a mode must sum to the
    oracle's whole field: a wrong permutation entry for one position would fail here."""
    rng = np.random.default_rng(7)
    if kind == "random":
        N = 14
        quads = pkg.fmc_graph(workload.random_frequencies(N, 91))
    elif kind == "comb":
        N = 12
        quads = oracle.enumerate_quads(N)
    else:
        N = 64
        quads = workload.sparse_comb_graph(N, 6, 5)
    J = rng.standard_normal(len(quads)) / N
    off, rec, recJ = pkg.graph_records(N, quads, J)
    a = np.sqrt(rng.uniform(0.3, 1.5, N)) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))
    J32 = J.astype(np.float32).astype(np.float64)
    splittings = set()
    for l in range(N):
        held = [q for q in range(len(quads)) if l in quads[q]]
        assert off[l + 1] - off[l] == len(held)
        tot = 0j
        for e, q in zip(range(off[l], off[l + 1]), held):
            A, B, C, w = (int(v) for v in rec[e])
            assert A % 8 == 0 and B % 8 == 0 and C % 8 == 0
            mA, mB, mC = A // 8, B // 8, C // 8
            pos, pA, pB, pC = w & 3, (w >> 2) & 3, (w >> 4) & 3, (w >> 6) & 3
            assert sorted([pos, pA, pB, pC]) == [0, 1, 2, 3]
            assert quads[q][pos] == l and quads[q][pA] == mA and quads[q][pB] == mB and quads[q][pC] == mC
            assert recJ[e] == np.float32(J[q])
            term = float(recJ[e]) * a[mA] * a[mB] * np.conj(a[mC])
            ref = oracle.field(N, quads[q:q + 1], J32[q:q + 1], a, l)
            assert abs(term - ref) <= 1e-12 * (abs(ref) + 1e-300), (l, q, pos, term, ref)
            splittings.add(pos)
            tot += term
        assert abs(tot - oracle.field(N, quads, J32, a, l)) <= 1e-11 * (abs(tot) + 1e-3)
    assert splittings == {0, 1, 2, 3}


def test_incidence_records_reject_bad_lists():
    with pytest.raises(pkg.PTError):
        pkg.graph_records(8, np.array([[0, 1, 2, 9]]), np.ones(1))
    with pytest.raises(pkg.PTError):
        pkg.graph_records(3, np.array([[0, 1, 2, 3]]), np.ones(1))
