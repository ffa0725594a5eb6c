"""Per-update parity of the production sweep kernel against the FP64 oracle.

pt_trace_update runs one sweep through the same kernel, block shape and CUDA graph as pt_sweep and has
the kernel record, for one pair update, what it reduced (h_j, h_k, B_jk, A_jk), its proposal, uniform,
Delta H and decision, and every chain's state just before the update.  Each record is checked element
by element against the oracle evaluated on that same state (Sec. III.A.1 pair move, Sec. III.A.3
parallel Delta E, cross term of reading R5):

  - (j, k) equal to the oracle's pair draw for (seed, sample, sweep, update);
  - h_j, h_k against or_field, B_jk and A_jk against or_cross_terms, within TOL x the magnitude of the
    sum (the larger of |value| and the root sum of squares of its terms);
  - the proposal and U against or_propose on the same state (FP32: the kernel draws in FP32);
  - Delta H against or_delta_h for the kernel's own proposal;
  - the decision against the oracle's Metropolis test, except where the two sides' Delta H straddle the
    threshold within the tolerance (counted, and bounded);
  - beta and, for FP64, the running energy against H(state).

Shapes: the N = 256 bench launch (16 samples x 48 T x 2 replicas, 8 chains x 11 field warps, packed FP32
blocks, B_jk gathered by the copy warp), N = 128 and 96 on 8 x 11 and on their 16-chain default (16 x 11), N = 64
on 32 x 7, 32 x 11 (its default) and 16 x 11, N = 48 on 8 chains (the gather threshold), N = 32 on 32 x 7, N = 24
on 8 x 7 and N = 16 on 16 x 7 (B picked out of the blocks), N = 4 (one quadruplet), N = 6 and the largest N = 512
(FP32 and FP64: the coupling ring then holds fewer stages), ragged batches with the
default and the autotuned shape (mixing the gathered and picked-out variants in one launch), and the FP64
kernels.  Updates include the first
and last of a sweep and pairs at the ends of the mode range, adjacent pairs and j + k = N - 1.
"""
import numpy as np
import pytest

import oracle
import paper_2511_13508_gb300 as pkg
from paper_2511_13508_gb300 import workload

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp64": 1e-12}
_QUADS = {}
WORST = {}  # largest relative errors seen per precision (printed at the end of the module, with -s)


@pytest.fixture(scope="module", autouse=True)
def _report():
    yield
    for prec, w in WORST.items():
        print("\ntrace %s: largest |GPU - oracle| / magnitude: fields %.2e, B/A %.2e, Delta H %.2e"
              % (prec, w["h"], w["BA"], w["dH"]))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def quads(N):
    if N not in _QUADS:
        _QUADS[N] = oracle.enumerate_quads(N)
    return _QUADS[N]


def couplings(Ns, seed0):
    return [workload.couplings(N, len(quads(N)), seed0 + s) for s, N in enumerate(Ns)]


def term_scale(q, J, x, modes):
    """Root sum of squares of the terms of the quadruplets holding every mode in `modes`, each term
    |J| times the magnitudes of the quadruplet's other factors."""
    m = np.ones(len(q), bool)
    for l in modes:
        m &= (q == l).any(1)
    qs, Js = q[m], J[m]
    mag = np.abs(x)[qs]
    for l in modes:
        mag = np.where(qs == l, 1.0, mag)
    return float(np.sqrt(((np.abs(Js) * mag.prod(1)) ** 2).sum()))


def state_offsets(Ns, R, nT):
    off, p = [], 0
    for N in Ns:
        for _ in range(R * nT):
            off.append(p); p += N
    return off


def check_records(rec, a, Ns, Js, temps, R, nT, seed, sweep, update, chains, prec):
    """Checks the trace records of `chains` (canonical ids); returns (checked, ambiguous decisions)."""
    tol = TOL[prec]
    off = state_offsets(Ns, R, nT)
    checked = ambiguous = 0
    worst = WORST.setdefault(prec, {"h": 0.0, "BA": 0.0, "dH": 0.0})
    for ci in chains:
        s, t = ci // (R * nT), ci % nT
        N = Ns[s]
        r_ = rec[ci]
        if update >= N // 2:
            assert r_[19] == 0.0, (ci, "record written past the sample's last update")
            continue
        assert r_[19] == 1.0, (ci, "no record")
        j, k = int(r_[0]), int(r_[1])
        assert (j, k) == oracle.pair(seed, s, sweep, update, N), (ci, j, k)
        x = a[off[ci]:off[ci] + N]
        q, J = quads(N), Js[s]
        hj, hk = complex(r_[2], r_[3]), complex(r_[4], r_[5])
        B, A = complex(r_[6], r_[7]), complex(r_[8], r_[9])
        hj_o, hk_o = oracle.field(N, q, J, x, j), oracle.field(N, q, J, x, k)
        B_o, A_o = oracle.cross_terms(N, q, J, x, j, k)
        sj, sk = term_scale(q, J, x, [j]), term_scale(q, J, x, [k])
        sjk = term_scale(q, J, x, [j, k])
        worst["h"] = max(worst["h"], abs(hj - hj_o) / max(abs(hj_o), sj), abs(hk - hk_o) / max(abs(hk_o), sk))
        worst["BA"] = max(worst["BA"], abs(B - B_o) / max(abs(B_o), sjk, 1e-300), abs(A - A_o) / max(abs(A_o), sjk, 1e-300))
        assert abs(hj - hj_o) <= tol * max(abs(hj_o), sj), (ci, j, k, hj, hj_o)
        assert abs(hk - hk_o) <= tol * max(abs(hk_o), sk), (ci, j, k, hk, hk_o)
        assert abs(B - B_o) <= tol * max(abs(B_o), sjk) + 1e-300, (ci, j, k, B, B_o)
        assert abs(A - A_o) <= tol * max(abs(A_o), sjk) + 1e-300, (ci, j, k, A, A_o)
        # proposal from the same Philox counters on the same state
        nj, nk, U = complex(r_[10], r_[11]), complex(r_[12], r_[13]), r_[14]
        nj_o, nk_o, U_o = oracle.propose(seed, ci, sweep, update, x, j, k)
        # intensities u = K^2 cos(theta), K^2 sin(theta) and phases are well conditioned in the drawn words
        # (the amplitudes sqrt(cos theta) are not, near theta = pi/2)
        K2 = (abs(x[j]) ** 4 + abs(x[k]) ** 4) ** 0.5
        ptol = 1e-6 if prec == "fp32" else 1e-13
        for n_, o_ in ((nj, nj_o), (nk, nk_o)):
            assert abs(abs(n_) ** 2 - abs(o_) ** 2) <= ptol * K2, (ci, n_, o_)
            assert abs(np.angle(n_ * np.conj(o_))) * abs(o_) <= ptol * np.sqrt(K2), (ci, n_, o_)
        assert abs(U - U_o) <= (1e-7 if prec == "fp32" else 1e-15), (ci, U, U_o)
        # Delta H of the kernel's own proposal
        dH, acc, beta = r_[15], r_[16], r_[17]
        dH_o = oracle.delta_h(N, q, J, x, j, k, nj, nk)
        dscale = abs(nj - x[j]) * sj + abs(nk - x[k]) * sk + abs(nj - x[j]) * abs(nk - x[k]) * sjk
        worst["dH"] = max(worst["dH"], abs(dH - dH_o) / max(abs(dH_o), dscale))
        assert abs(dH - dH_o) <= tol * max(abs(dH_o), dscale), (ci, dH, dH_o, dscale)
        assert beta == pytest.approx(1.0 / temps[t], rel=1e-7 if prec == "fp32" else 1e-15)
        acc_o = dH_o <= 0.0 or U_o < np.exp(-beta * dH_o)
        # the decision is fixed unless the threshold lies within the tolerance of both sides' Delta H
        margin = tol * max(abs(dH_o), dscale) * 4
        near = abs(dH_o) <= margin or (U_o > 0 and abs(-np.log(U_o) / max(beta, 1e-300) - dH_o) <= margin)
        if near:
            ambiguous += 1
        else:
            assert bool(acc) == bool(acc_o), (ci, dH, dH_o, U, beta, acc)
        if prec == "fp64":
            E_o = oracle.energy(N, q, J, x)
            assert abs(r_[18] - E_o) <= 1e-9 * (abs(E_o) + 1.0), (ci, r_[18], E_o)
        checked += 1
    return checked, ambiguous


def pick_updates(seed, Ns, sweep, n_pick=3):
    """Updates of `sweep` whose pair (in some sample) touches an end of the mode range, is adjacent, or has
    j + k = N - 1; plus the first and last update.  Returns [(update, [samples showing it])]."""
    maxu = max(Ns) // 2
    cats = {"end": [], "adjacent": [], "mid-sum": []}
    for u in range(maxu):
        for s, N in enumerate(Ns):
            if u >= N // 2:
                continue
            j, k = oracle.pair(seed, s, sweep, u, N)
            if min(j, k) == 0 or max(j, k) == N - 1:
                cats["end"].append((u, s))
            if abs(j - k) == 1:
                cats["adjacent"].append((u, s))
            if j + k == N - 1:
                cats["mid-sum"].append((u, s))
    picks = []
    for name in ("end", "adjacent", "mid-sum"):
        if cats[name]:
            u = cats[name][0][0]
            picks.append((u, sorted({s for uu, s in cats[name] if uu == u})))
    return picks[:n_pick]


def run_traces(pt, Ns, Js, temps, R, nT, seed, prec, n_calls, chains_per_sample=4, samples=None):
    """n_calls traced sweeps: the first traces update 0, the second the last update of the largest N, the
    rest the edge-case updates picked from the pair sequence.  Checks a few chains of the samples concerned."""
    rng = np.random.default_rng(seed)
    cps = R * nT
    tot = amb = 0
    for call in range(n_calls):
        sweep = pt.counters[0]
        if call == 0:
            u, ss = 0, list(range(len(Ns)))
        elif call == 1:
            u, ss = max(Ns) // 2 - 1, list(range(len(Ns)))
        else:
            picks = pick_updates(seed, Ns, sweep)
            u, ss = picks[(call - 2) % len(picks)] if picks else (0, list(range(len(Ns))))
        if samples is not None:
            ss = [s for s in ss if s in samples] or [samples[0]]
        rec, a = pt.trace_update(u)
        assert pt.counters[0] == sweep + 1
        written = rec[:, 19] == 1.0
        expect = np.array([u < Ns[ci // cps] // 2 for ci in range(len(rec))])
        assert np.array_equal(written, expect)
        chains = []
        for s in ss:
            sel = rng.choice(cps, size=min(chains_per_sample, cps), replace=False)
            chains += [s * cps + int(c) for c in sel]
        n, m = check_records(rec, a, Ns, Js, temps, R, nT, seed, sweep, u, chains, prec)
        tot += n; amb += m
    assert tot > 0
    assert amb <= max(1, tot // 20), (amb, tot)
    return tot


CASES = [
    # name, Ns, R, nT, precision, chains_per_block, consumer_warps
    ("n128_8x11_gatherB", [128, 128], 2, 6, "fp32", 8, 11),
    ("n128_default_16chains", [128, 128], 2, 8, "fp32", 0, 0),
    ("n96_8x11_gatherB", [96, 96], 2, 5, "fp32", 8, 11),
    ("n96_default_16chains", [96, 96], 2, 8, "fp32", 0, 0),
    ("n64_32x7", [64, 64], 2, 16, "fp32", 32, 7),
    ("n64_default_32x11", [64, 64], 2, 16, "fp32", 0, 0),
    ("n64_16x11", [64, 64], 2, 8, "fp32", 16, 11),
    ("n48_8chains_packed", [48, 48, 48], 2, 5, "fp32", 8, 0),
    ("n32_32x7_picked_B", [32, 32], 2, 16, "fp32", 32, 7),
    ("n16_16x7", [16, 16], 2, 8, "fp32", 0, 0),
    ("n4_single_quadruplet", [4, 4, 4], 2, 3, "fp32", 0, 0),
    ("n6_fp64", [6, 6], 2, 3, "fp64", 0, 0),
    ("n24_8x7_packed", [24, 24], 2, 4, "fp32", 0, 0),
    ("ragged_mixed", [128, 32, 96, 48, 64, 96, 32], 2, 6, "fp32", 0, 0),
    ("n64_fp64_16x3", [64, 64], 2, 5, "fp64", 0, 0),
    ("n128_fp64_8x7", [128], 2, 4, "fp64", 0, 0),
    ("ragged_fp64", [40, 24, 64], 2, 3, "fp64", 0, 0),
    ("n512_largest_fp32", [512], 2, 2, "fp32", 0, 0),
    ("n512_largest_fp64", [512], 1, 2, "fp64", 0, 0),
]


@pytest.mark.parametrize("name,Ns,R,nT,prec,cpb,cw", CASES, ids=[c[0] for c in CASES])
def test_trace_matches_oracle(name, Ns, R, nT, prec, cpb, cw):
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns, 5000 + len(Ns))
    seed = 4242
    pt = pkg.PT(Ns, Js, temps, R, seed, precision=prec, chains_per_block=cpb, consumer_warps=cw,
                swap_every=8, measure_every=4, resync_every=16)
    pt.sweep(21)  # off the beta = 0 start, through swaps, resyncs and measurements
    run_traces(pt, Ns, Js, temps, R, nT, seed, prec, n_calls=5)


def test_trace_ragged_autotuned_shape():
    Ns, R, nT = [128, 48, 96, 64, 32, 96, 128, 48], 2, 6
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns, 6100)
    pt = pkg.PT(Ns, Js, temps, R, 77, precision="fp32", swap_every=8, measure_every=4, resync_every=16)
    pt.autotune(trial_sweeps=2)
    pt.sweep(9)
    run_traces(pt, Ns, Js, temps, R, nT, 77, "fp32", n_calls=4)


def test_trace_n256_bench_launch():
    """The bench's N = 256 launch itself: 16 samples x 48 T x 2 replicas, default shape, CUDA graphs."""
    W = workload.workloads()["n256_large"]
    N = 256
    Js = [workload.couplings(N, len(quads(N)), s) for s in W.seeds]
    pt = pkg.PT(W.Ns, Js, W.temps, W.replicas, 12345, precision="fp32", swap_every=W.swap_every,
                measure_every=W.measure_every, resync_every=W.resync_every)
    pt.sweep(66)  # past a swap pass and a resync
    run_traces(pt, list(W.Ns), Js, W.temps, W.replicas, len(W.temps), 12345, "fp32", n_calls=5,
               chains_per_sample=3, samples=[0, 5, 15])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_trace_sweep_equals_plain_sweep(prec):
    """A traced sweep is the same sweep: two contexts with the same seed, one advanced by pt_trace_update and
    one by pt_sweep, hold bit-identical states, energies and counters."""
    Ns, R, nT = [64, 32], 2, 6
    temps = workload.geometric_ladder(0.3, 1.6, nT)
    Js = couplings(Ns, 7000)
    kw = dict(precision=prec, swap_every=4, measure_every=2, resync_every=8)
    a = pkg.PT(Ns, Js, temps, R, 9, **kw)
    b = pkg.PT(Ns, Js, temps, R, 9, **kw)
    for it in range(9):  # crosses measurement, swap and resync points
        a.trace_update(it % 16)
        b.sweep(1)
    sa, Ea = a.state()
    sb, Eb = b.state()
    assert np.array_equal(sa, sb) and np.array_equal(Ea, Eb)
    oa, ob = a.observables(), b.observables()
    for key in oa:
        assert np.array_equal(oa[key], ob[key]), key


def test_trace_arguments():
    Js = couplings([16], 7100)
    pt = pkg.PT([16], Js, [0.5, 1.0], 2, 1)
    with pytest.raises(pkg.PTError) as e:
        pt.trace_update(8)
    assert e.value.code == -1
    with pytest.raises(pkg.PTError):
        pt.trace_update(-1)
    pp = pkg.PT([16], Js, [0.5, 1.0], 2, 1, precision="fp64_plain")
    with pytest.raises(pkg.PTError) as e:
        pp.trace_update(0)
    assert e.value.code == -7
