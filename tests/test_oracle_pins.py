"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle function to something other than itself: published
known-answer vectors, brute force, closed forms derived from the paper's target law
(Eq. (8): P[a] ~ exp(-beta H) delta(N - sum |a|^4)), exact symmetries of Eq. (4),
independent exact sampling at beta = 0 with importance reweighting, and N = 4
quadrature.  None of these recomputes the oracle's own formula.
"""
import itertools
import math
import os

import numpy as np
import pytest
from scipy import special

import oracle
from paper_2511_13508_gb300 import workload

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_state(N, rng, on_constraint=True):
    g = rng.standard_normal(N)
    u = np.sqrt(N) * np.abs(g) / np.linalg.norm(g) if on_constraint else rng.uniform(0.2, 1.5, N)
    return np.sqrt(u) * np.exp(1j * rng.uniform(0, 2 * np.pi, N))


def exact_beta0_samples(N, n, rng):
    """Independent exact draws of the beta = 0 law: u uniform on {u >= 0, sum u^2 = N}, phases uniform."""
    g = rng.standard_normal((n, N))
    u = np.sqrt(N) * np.abs(g) / np.linalg.norm(g, axis=1, keepdims=True)
    return np.sqrt(u) * np.exp(1j * rng.uniform(0, 2 * np.pi, (n, N)))


# ------------------------------------------------------------------------------------ RNG
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        assert oracle.philox(v[0:4], v[4:6]) == v[6:10]


def test_uniform_open_interval():
    assert oracle.lib().or_uniform(0) == 0.5 / 2 ** 32
    assert oracle.lib().or_uniform(0xffffffff) == (2 ** 32 - 0.5) / 2 ** 32 < 1.0


# ------------------------------------------------------------------------------------ graph
@pytest.mark.parametrize("N", [4, 5, 6, 7, 8, 11, 14])
def test_quads_bruteforce(N):
    """Quadruplets of the comb (distinct modes, a+d=b+c) by brute force over all 4-subsets."""
    brute = [q for q in itertools.combinations(range(N), 4) if q[0] + q[3] == q[1] + q[2]]
    got = [tuple(int(x) for x in q) for q in oracle.enumerate_quads(N)]
    assert got == brute  # same set, lexicographic order


@pytest.mark.parametrize("N", [16, 64, 128, 256])
def test_quad_counts_closed_form(N):
    """|Q| = sum_s C(m_s, 2), m_s = number of pairs {x < y} with x + y = s (the pairs sharing a sum)."""
    m = np.array([sum(1 for x in range(N) if x < s - x < N) for s in range(2 * N)])
    assert len(oracle.enumerate_quads(N)) == int((m * (m - 1) // 2).sum())


def test_connectivity_ratio_tends_to_paper_value():
    """c_FMC / c_fc -> (1 + 2N^2)/N^3 ~ 2/N (Eq. (9)); on the integer comb the relative gap shrinks with N."""
    gaps = []
    for N in (32, 64, 128, 256):
        m = np.array([sum(1 for x in range(N) if x < s - x < N) for s in range(2 * N)])
        ratio = (m * (m - 1) // 2).sum() / math.comb(N, 4)
        gaps.append(abs(ratio / ((1 + 2 * N * N) / N ** 3) - 1))
    assert gaps[-1] < 0.01 and all(g1 < g0 for g0, g1 in zip(gaps, gaps[1:]))


# ------------------------------------------------------------------------------------ Hamiltonian
def test_single_quadruplet_closed_form():
    """N = 4 has the single quadruplet (0,1,2,3): H = -2 J A0 A1 A2 A3 cos(phi1 + phi2 - phi0 - phi3)."""
    rng = np.random.default_rng(1)
    q = oracle.enumerate_quads(4)
    assert q.tolist() == [[0, 1, 2, 3]]
    for _ in range(20):
        A = rng.uniform(0.1, 2.0, 4); ph = rng.uniform(0, 2 * np.pi, 4); J = rng.standard_normal(1)
        a = A * np.exp(1j * ph)
        ref = -2.0 * J[0] * A.prod() * np.cos(ph[1] + ph[2] - ph[0] - ph[3])
        assert oracle.energy(4, q, J, a) == pytest.approx(ref, rel=1e-13, abs=1e-15)


@pytest.mark.parametrize("N", [8, 13, 24])
def test_energy_gauge_invariances(N):
    """H(e^{i alpha} a) = H(a) (global phase) and H(a_k e^{i k theta}) = H(a) (comb/FMC gauge)."""
    rng = np.random.default_rng(N)
    q = oracle.enumerate_quads(N); J = rng.standard_normal(len(q)) / N
    a = rand_state(N, rng)
    E = oracle.energy(N, q, J, a)
    for alpha in rng.uniform(0, 2 * np.pi, 3):
        assert oracle.energy(N, q, J, a * np.exp(1j * alpha)) == pytest.approx(E, rel=1e-13)
        assert oracle.energy(N, q, J, a * np.exp(1j * alpha * np.arange(N))) == pytest.approx(E, rel=1e-13)
    # a gauge that is NOT a symmetry must change H (guards against a trivially invariant H)
    assert abs(oracle.energy(N, q, J, a * np.exp(1j * 0.7 * np.arange(N) ** 2)) - E) > 1e-3 * abs(E)


def test_energy_brute_force_sum():
    """H = -2 sum over all ordered index 4-tuples satisfying the FMC, each unordered quadruplet once."""
    rng = np.random.default_rng(7)
    N = 7
    q = oracle.enumerate_quads(N); J = rng.standard_normal(len(q))
    a = rand_state(N, rng, on_constraint=False)
    Jd = {tuple(x): J[i] for i, x in enumerate(q.tolist())}
    tot = 0.0
    for k1, k2, k3, k4 in itertools.permutations(range(N), 4):
        # term conj(a_k1) a_k2 conj(a_k3) a_k4 with omega_k1 - omega_k2 + omega_k3 - omega_k4 = 0
        if k1 - k2 + k3 - k4 != 0:
            continue
        key = tuple(sorted((k1, k2, k3, k4)))
        tot += Jd[key] * (np.conj(a[k1]) * a[k2] * np.conj(a[k3]) * a[k4]).real
    # each quadruplet appears 8 times among ordered tuples (2 pairings x 2 x 2 orders); "+ c.c." doubles
    assert oracle.energy(N, q, J, a) == pytest.approx(-2.0 * tot / 8.0, rel=1e-12)


@pytest.mark.parametrize("N", [6, 12, 20])
def test_field_is_exact_single_mode_derivative(N):
    """H is multilinear in (a_l, conj a_l), so H(a_l + d) - H(a) = -2 Re(conj(d) h_l) exactly."""
    rng = np.random.default_rng(100 + N)
    q = oracle.enumerate_quads(N); J = rng.standard_normal(len(q)) / N
    a = rand_state(N, rng)
    E = oracle.energy(N, q, J, a)
    for l in range(N):
        d = complex(*rng.standard_normal(2))
        b = a.copy(); b[l] += d
        h = oracle.field(N, q, J, a, l)
        assert oracle.energy(N, q, J, b) - E == pytest.approx(-2.0 * (np.conj(d) * h).real, rel=1e-10, abs=1e-13)


@pytest.mark.parametrize("N", [4, 6, 9, 16, 32])
def test_delta_h_matches_full_recompute(N):
    """Pair-update Delta H (two fields + j-k cross term) equals H(a') - H(a) recomputed in full."""
    rng = np.random.default_rng(200 + N)
    q = oracle.enumerate_quads(N); J = rng.standard_normal(len(q)) / N
    a = rand_state(N, rng)
    E = oracle.energy(N, q, J, a)
    worst = 0.0
    for _ in range(60):
        j, k = rng.choice(N, 2, replace=False)
        ajn, akn = complex(*rng.standard_normal(2)), complex(*rng.standard_normal(2))
        b = a.copy(); b[j] = ajn; b[k] = akn
        full = oracle.energy(N, q, J, b) - E
        dh = oracle.delta_h(N, q, J, a, j, k, ajn, akn)
        worst = max(worst, abs(dh - full) / max(abs(full), 1e-12))
    assert worst < 1e-11


@pytest.mark.parametrize("N", [4, 7, 10, 16, 24])
def test_cross_terms_complete_the_pair_change(N):
    """H is multilinear in the factors of every quadruplet, so for a_j += dj, a_k += dk the change is exactly
    -2 Re[conj(dj) h_j + conj(dk) h_k + conj(dj) dk B + conj(dj) conj(dk) A]: full recompute for several
    independent (dj, dk) per pair determines B and A, so a swapped, conjugated or dropped term fails."""
    rng = np.random.default_rng(300 + N)
    q = oracle.enumerate_quads(N); J = rng.standard_normal(len(q)) / N
    a = rand_state(N, rng, on_constraint=False)
    E = oracle.energy(N, q, J, a)
    pairs = [(0, N - 1), (N - 1, 0), (0, 1), (1, 0), (N // 2 - 1, N // 2)] + \
        [tuple(rng.choice(N, 2, replace=False)) for _ in range(6)]
    for j, k in pairs:
        hj, hk = oracle.field(N, q, J, a, j), oracle.field(N, q, J, a, k)
        B, A = oracle.cross_terms(N, q, J, a, j, k)
        for _ in range(4):
            dj, dk = complex(*rng.standard_normal(2)), complex(*rng.standard_normal(2))
            b = a.copy(); b[j] += dj; b[k] += dk
            full = oracle.energy(N, q, J, b) - E
            dec = -2.0 * (np.conj(dj) * hj + np.conj(dk) * hk + np.conj(dj) * dk * B + np.conj(dj) * np.conj(dk) * A).real
            assert dec == pytest.approx(full, rel=1e-10, abs=1e-12), (j, k)


def test_cross_terms_single_quadruplet_closed_form():
    """N = 4, quadruplet (0,1,2,3), term J conj(a0) a1 a2 conj(a3): both modes of one pair give A = J times the
    other pair's plain product; modes of different pairs give B = J conj(m) y with j+m = k+y."""
    rng = np.random.default_rng(5)
    q = oracle.enumerate_quads(4); J = np.array([0.7])
    a = rand_state(4, rng, on_constraint=False)
    c = np.conj
    cases = {(0, 3): (0.0, 0.7 * a[1] * a[2]), (1, 2): (0.0, 0.7 * a[0] * a[3]),
             (0, 1): (0.7 * c(a[3]) * a[2], 0.0), (0, 2): (0.7 * c(a[3]) * a[1], 0.0),
             (1, 0): (0.7 * c(a[2]) * a[3], 0.0), (2, 3): (0.7 * c(a[1]) * a[0], 0.0)}
    for (j, k), (Bref, Aref) in cases.items():
        B, A = oracle.cross_terms(4, q, J, a, j, k)
        assert abs(B - Bref) < 1e-14 and abs(A - Aref) < 1e-14, (j, k, B, Bref, A, Aref)


# ------------------------------------------------------------------------------------ move
def test_pair_draw_distribution():
    """j uniform on [0,N), k uniform on the other N-1 modes (chi-square on the joint counts)."""
    N = 6
    counts = np.zeros((N, N))
    for u in range(30000):
        j, k = oracle.pair(12345, 3, 7, u, N)
        assert j != k and 0 <= j < N and 0 <= k < N
        counts[j, k] += 1
    exp = 30000 / (N * (N - 1))
    off = ~np.eye(N, dtype=bool)
    chi2 = ((counts[off] - exp) ** 2 / exp).sum()
    assert counts[~off].sum() == 0
    assert chi2 < 60  # 29 dof: p ~ 5e-4


def test_proposal_preserves_pair_quartic_and_law():
    """|a_j'|^4 + |a_k'|^4 = K^4 exactly; theta uniform on [0, pi/2]; phases uniform (Sec. III.A.1)."""
    rng = np.random.default_rng(3)
    N = 10
    a = rand_state(N, rng)
    thetas = []
    for u in range(4000):
        j, k = 2, 7
        aj, ak, U = oracle.propose(99, 5, 1, u, a, j, k)
        K4 = abs(a[j]) ** 4 + abs(a[k]) ** 4
        assert abs(aj) ** 4 + abs(ak) ** 4 == pytest.approx(K4, rel=1e-13)
        thetas.append(math.atan2(abs(ak) ** 2, abs(aj) ** 2))  # |aj|^2 = K^2 cos, |ak|^2 = K^2 sin
        assert 0 < U < 1
    h, _ = np.histogram(thetas, bins=10, range=(0, np.pi / 2))
    assert ((h - 400) ** 2 / 400).sum() < 35


def test_init_on_constraint_surface():
    for N in (4, 16, 64):
        for c in range(5):
            a = oracle.init_config(7, c, N)
            assert (np.abs(a) ** 4).sum() == pytest.approx(N, rel=1e-14)


# ------------------------------------------------------------------------------------ observables
def test_observables_on_hand_built_states():
    N = 16
    a = np.exp(1j * np.linspace(0, 3, N))  # |a_k| = 1 -> sum |a|^4 = N
    assert oracle.ipr(a, 2) == pytest.approx(1.0 / N, rel=1e-14)
    assert oracle.ipr(a, 4) == pytest.approx(1.0 / N, rel=1e-14)
    assert oracle.overlap(a, a) == pytest.approx(1.0, rel=1e-14)       # q(a,a) = I/N
    assert oracle.overlap(a, -a) == pytest.approx(-1.0, rel=1e-14)
    b = a * np.where(np.arange(N) % 2 == 0, 1j, 1.0)
    assert oracle.overlap(a, b) == pytest.approx(0.5, rel=1e-14)
    c = np.zeros(N, complex); c[3] = N ** 0.25                        # fully condensed
    assert oracle.ipr(c, 2) == pytest.approx(1.0) and oracle.ipr(c, 4) == pytest.approx(1.0)
    assert [oracle.qbin(x) for x in (-1.0, -0.995, -0.9949, 0.0, 0.004, 0.006, 1.0, 1.5)] == \
        [0, 1, 1, 100, 100, 101, 200, 200]


# ------------------------------------------------------------------------------------ engine
def make_pt(N, S, temps, R, seed, **kw):
    Js = [workload.couplings(N, len(oracle.enumerate_quads(N)), 1000 + s) for s in range(S)]
    return oracle.OraclePT([N] * S, Js, temps, R, seed, **kw), Js


def test_constraint_and_running_energy_over_2048_sweeps():
    """FP64, no resync: sum|a|^4 stays N to 1e-12 N and the tracked E equals the full H to 1e-10."""
    N = 16
    pt, Js = make_pt(N, 2, workload.geometric_ladder(0.4, 1.6, 4), 2, 11, resync_every=0, measure_every=0)
    pt.sweep(2048)
    a, E = pt.state()
    a = a.reshape(-1, N)
    q = oracle.enumerate_quads(N)
    for c in range(a.shape[0]):
        assert abs((np.abs(a[c]) ** 4).sum() - N) <= 1e-12 * N
        s = c // (2 * 4)
        assert E[c] == pytest.approx(oracle.energy(N, q, Js[s], a[c]), rel=1e-10, abs=1e-12)


def test_beta_zero_law_is_preserved():
    """At beta = 0 the move keeps the uniform law on the constraint surface:
    <Y4> = 3/(N+2), <I> = N^{3/2} G(N/2)/(sqrt(pi) G((N+1)/2)), <q^2> = G(N/2)^2/(2 pi G((N+1)/2)^2), <H> = 0."""
    N = 8
    pt, _ = make_pt(N, 1, [1e12], 24, 5, swap_every=0, measure_every=4, resync_every=0)
    pt.sweep(200)
    pt.reset_observables()
    pt.sweep(20000)
    o = pt.observables()
    st, qs = o["stat"][0, 0], o["qstat"][0, 0]
    n = st[0]
    y4 = st[4] / n
    I = st[5] / n
    q2 = qs[2] / qs[0]
    ref_y4 = 3.0 / (N + 2)
    ref_I = N ** 1.5 * math.exp(math.lgamma(N / 2) - math.lgamma((N + 1) / 2)) / math.sqrt(math.pi)
    ref_q2 = math.exp(2 * (math.lgamma(N / 2) - math.lgamma((N + 1) / 2))) / (2 * math.pi)
    # statistical tolerances from exact beta=0 sampling of the same number of effectively independent draws
    rng = np.random.default_rng(0)
    x = exact_beta0_samples(N, 200000, rng)
    sd_y4 = ((np.abs(x) ** 8).sum(1) / N ** 2).std()
    sd_I = (np.abs(x) ** 2).sum(1).std()
    neff = n / 8  # conservative: correlation time <= 8 measurements at beta = 0
    assert abs(y4 - ref_y4) < 4 * sd_y4 / math.sqrt(neff)
    assert abs(I - ref_I) < 4 * sd_I / math.sqrt(neff)
    assert abs(q2 - ref_q2) < 4 * ref_q2 * math.sqrt(2) / math.sqrt(qs[0] / 8)
    assert abs(st[1] / n) < 4 * math.sqrt(st[2] / n) / math.sqrt(neff)
    # and the closed forms themselves against exact sampling (pins the derivation)
    assert np.mean((np.abs(x) ** 8).sum(1)) / N ** 2 == pytest.approx(ref_y4, rel=0.01)
    assert np.mean((np.abs(x) ** 2).sum(1)) == pytest.approx(ref_I, rel=0.003)


def test_small_beta_energy_by_reweighting():
    """<H>_beta of the chain equals E0[H e^{-beta H}] / E0[e^{-beta H}] from exact beta=0 draws, and
    Var_0(H) = (8N / (pi^2 (N+2))) sum_q J_q^2 (cc = 2), so <H>_beta ~ -beta Var_0(H) at small beta."""
    N = 12
    q = oracle.enumerate_quads(N)
    temps = [10.0, 3.0]
    pt, Js = make_pt(N, 1, temps, 16, 21, swap_every=0, measure_every=2, resync_every=0)
    pt.sweep(500); pt.reset_observables(); pt.sweep(12000)
    st = pt.observables()["stat"][0]
    rng = np.random.default_rng(1)
    x = exact_beta0_samples(N, 60000, rng)
    H0 = np.array([oracle.energy(N, q, Js[0], xi) for xi in x])
    var0 = (8 * N / (math.pi ** 2 * (N + 2))) * (Js[0] ** 2).sum()
    assert H0.var() == pytest.approx(var0, rel=0.03)
    for t, T in enumerate(temps):
        b = 1.0 / T
        w = np.exp(-b * (H0 - H0.mean()))
        ref = (H0 * w).sum() / w.sum()
        chain = st[t, 1] / st[t, 0]
        sd = math.sqrt(st[t, 2] / st[t, 0] - chain ** 2)
        err = sd / math.sqrt(st[t, 0] / 10) + 3 * H0.std() / math.sqrt(len(H0))
        assert abs(chain - ref) < 4 * err, (T, chain, ref, err)
        assert ref == pytest.approx(-b * var0, rel=0.25)


def _n4_quadrature(J, betas, n=2_000_000, seed=0):
    """N = 4 single quadruplet.  Integrating the relative phase gives Z ~ E_u[I0(2 beta J w)], w = sqrt(u0 u1 u2 u3),
    u uniform on the positive orthant of sum u^2 = 4, so <E> = -E_u[2 J w I1(2 beta J w)] / E_u[I0(2 beta J w)]."""
    rng = np.random.default_rng(seed)
    g = np.abs(rng.standard_normal((n, 4)))
    u = 2.0 * g / np.linalg.norm(g, axis=1, keepdims=True)
    w = np.sqrt(u.prod(1))
    out = []
    for b in betas:
        x = 2 * b * J * w
        i0 = special.i0e(x) * np.exp(np.abs(x) - np.abs(x).max())
        i1 = special.i1e(x) * np.exp(np.abs(x) - np.abs(x).max())
        out.append(-(2 * J * w * i1).sum() / i0.sum())
    return np.array(out)


def test_n4_chain_matches_quadrature_with_swaps():
    """The full PT engine (moves + swaps) at N = 4 reproduces <E>(beta) from quadrature within 4 sigma."""
    N = 4
    temps = np.array([0.05, 0.1, 0.2, 0.5])
    J = np.array([0.8])
    pt = oracle.OraclePT([N], [J], temps, 8, 77, swap_every=4, measure_every=2, resync_every=0)
    pt.sweep(2000); pt.reset_observables(); pt.sweep(60000)
    o = pt.observables()
    st = o["stat"][0]
    ref = _n4_quadrature(J[0], 1.0 / temps)
    for t in range(len(temps)):
        m = st[t, 1] / st[t, 0]
        sd = math.sqrt(st[t, 2] / st[t, 0] - m * m)
        err = sd / math.sqrt(st[t, 0] / 20)
        assert abs(m - ref[t]) < 4 * err + 2e-3 * abs(ref[t]), (temps[t], m, ref[t], err)
    assert (o["swap_acc"] > 0).all()


def test_n4_swap_acceptance_detailed_balance():
    """Two temperatures at N = 4: the swap acceptance rate equals E_{b1} E_{b2}[min(1, e^{(b1-b2)(E1-E2)})]
    computed from exact beta = 0 draws reweighted to each temperature (Eq. (15))."""
    N = 4
    temps = np.array([0.15, 0.3])
    J = np.array([0.7])
    pt = oracle.OraclePT([N], [J], temps, 16, 31, swap_every=8, measure_every=0, resync_every=0)
    pt.sweep(800); pt.reset_observables(); pt.sweep(48000)
    o = pt.observables()
    rate = o["swap_acc"].sum() / o["swap_att"].sum()
    rng = np.random.default_rng(5)
    x = exact_beta0_samples(N, 400000, rng)
    E0 = -2 * J[0] * (np.conj(x[:, 0]) * x[:, 1] * x[:, 2] * np.conj(x[:, 3])).real
    b1, b2 = 1 / temps
    w1 = np.exp(-b1 * (E0 - E0.min())); w1 /= w1.sum()
    w2 = np.exp(-b2 * (E0 - E0.min())); w2 /= w2.sum()
    i1 = rng.choice(len(E0), 200000, p=w1); i2 = rng.choice(len(E0), 200000, p=w2)
    ref = np.minimum(1.0, np.exp((b1 - b2) * (E0[i1] - E0[i2]))).mean()
    n = o["swap_att"].sum()
    assert abs(rate - ref) < 4 * math.sqrt(ref * (1 - ref) / (n / 4)) + 0.004, (rate, ref)
