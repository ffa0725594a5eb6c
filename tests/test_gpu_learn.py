"""Learned global-move proposal: tensor-core GEMM, network forward/backward and the exact MH move,
through the C ABI, against plain FP32/FP64 references."""
import ctypes
import math

import numpy as np
import pytest

import paper_2511_13508_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


@pytest.mark.parametrize("batch,M,N,K", [(1, 128, 256, 64), (3, 200, 256, 192), (2, 77, 192, 256),
                                         (1, 300, 64, 520), (2, 129, 16, 24), (1, 512, 256, 512)])
def test_tcgen05_gemm_matches_fp32_reference(batch, M, N, K):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * N + K)
    A = torch.randn(batch, M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(batch, N, K, device="cuda", generator=g).to(torch.bfloat16)
    D = torch.full((batch, M, N), float("nan"), device="cuda", dtype=torch.float32)
    L = pkg.lib()
    L.pt_gemm_bf16.argtypes = [ctypes.c_int] * 4 + [ctypes.c_void_p] * 4
    s = torch.cuda.current_stream()
    rc = L.pt_gemm_bf16(batch, M, N, K, A.data_ptr(), B.data_ptr(), D.data_ptr(), s.cuda_stream)
    assert rc == 0, L.pt_last_error(None)
    torch.cuda.synchronize()
    ref = torch.bmm(A.float(), B.float().transpose(1, 2))
    err = (D - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item() + 1e-4, err


# ------------------------------------------------------------------------------ learned proposal
from oracle import learned as ol  # noqa: E402
from paper_2511_13508_gb300 import workload  # noqa: E402


def _couplings(Ns, seed0=2000):
    import oracle
    return [workload.couplings(N, len(oracle.enumerate_quads(N)), seed0 + s) for s, N in enumerate(Ns)]


def _dirichlet(N, shape, alpha, rng):
    g = rng.gamma(alpha, size=shape + (N,))
    s = g / g.sum(-1, keepdims=True)
    return (N * s) ** 0.25 * np.exp(1j * rng.uniform(0, 2 * np.pi, shape + (N,)))


def _stick_breaking_biases(N, P, sh, s_rows=None):
    """Output biases near the stick-breaking law of Dirichlet(1/2) (the beta = 0 law), phases near uniform."""
    from scipy import special
    k = np.arange(N)
    b = np.maximum((N - k - 1) / 2, 0.5)
    b3 = np.zeros((N, 4))
    b3[:, 0] = special.digamma(0.5) - special.digamma(b)
    b3[:, 1] = 0.5 * np.log(special.polygamma(1, 0.5) + special.polygamma(1, b))
    b3[:, 3] = -6.0
    P[:, sh["ob3"]:sh["ob3"] + 4 * N] = b3.ravel()
    return P


def _randomise_outputs(P, sh, rng, scale=1.0):
    """Non-trivial output layer so that every term of the density is exercised."""
    S = P.shape[0]
    H, Dout = sh["H"], sh["Dout"]
    P[:, sh["oW3"]:sh["ob3"]] = scale * rng.uniform(-1, 1, (S, Dout * H)) / math.sqrt(H)
    b3 = np.zeros((S, Dout // 4, 4))
    b3[..., 0] = rng.normal(-1.0, 0.5, b3.shape[:2])
    b3[..., 1] = rng.normal(0.0, 0.3, b3.shape[:2])
    b3[..., 2] = rng.uniform(0, 2 * np.pi, b3.shape[:2])
    b3[..., 3] = rng.normal(0.0, 1.0, b3.shape[:2])
    P[:, sh["ob3"]:sh["ob3"] + Dout] = b3.reshape(S, Dout)
    P[:, sh["oC1"]:sh["oW2"]] = 0.2 * rng.standard_normal((S, sh["oW2"] - sh["oC1"]))
    return P


@pytest.mark.parametrize("N,rows", [(16, 200), (32, 128), (48, 72), (64, 256)])
def test_learn_eval_matches_oracle(N, rows):
    """Features, network (tcgen05 GEMMs) and density of the proposal against the FP64 oracle with the
    BF16 rounding points emulated; gradient of the mean NLL against the oracle's autograd gradient."""
    S, R, nT, ncold = 2, 8, 4, 3
    temps = workload.geometric_ladder(0.5, 1.5, nT)
    pt = pkg.PT([N] * S, _couplings([N] * S), temps, R, 5, precision="fp32")
    pt.learn_init(n_cold=ncold, batch=256, data_per_sample=256, seed=9)
    sh = pt.learn_shape()
    rng = np.random.default_rng(N + rows)
    P = _randomise_outputs(pt.learn_params().astype(np.float64), sh, rng).astype(np.float32)
    pt.set_learn_params(P)
    assert np.array_equal(pt.learn_params(), P)
    a = _dirichlet(N, (S, rows), 0.5, rng).astype(np.complex64).astype(np.complex128)
    cond = rng.integers(0, ncold, (S, rows)).astype(np.int32)
    lq, ex, g = pt.learn_eval(a, cond, grad=True)
    M1, M2, M3 = ol.masks(N, sh["H"], 8)
    for s in range(S):
        Ps = P[s].astype(np.float64)
        lq_o, ex_o = ol.logq(Ps, a[s], cond[s], N, sh["H"], ncold, 8, emulate_bf16=True)
        assert np.abs(ex[s] - ex_o).max() <= 1e-5 * np.abs(ex_o).max() + 1e-4
        err = np.abs(lq[s] - lq_o)
        assert err.max() <= 2e-3 + 1e-5 * np.abs(lq_o).max(), (err.max(), np.abs(lq_o).max())
        go, _ = ol.nll_grad(Ps, a[s], cond[s], N, sh["H"], ncold, 8, emulate_bf16=True)
        gg = g[s].astype(np.float64)
        parts = {"W1": (sh["oW1"], sh["ob1"], M1), "b1": (sh["ob1"], sh["oC1"], None), "C1": (sh["oC1"], sh["oW2"], None),
                 "W2": (sh["oW2"], sh["ob2"], M2), "b2": (sh["ob2"], sh["oW3"], None), "W3": (sh["oW3"], sh["ob3"], M3),
                 "b3": (sh["ob3"], sh["ob3"] + sh["Dout"], None)}
        for name, (lo, hi, M) in parts.items():
            x, y = gg[lo:hi], go[lo:hi]
            if M is not None:
                x = x * M.ravel()
            rel = np.linalg.norm(x - y) / (np.linalg.norm(y) + 1e-30)
            assert rel < 3e-2, (name, rel)


@pytest.mark.parametrize("N", [16, 64])
def test_learn_eval_geometric_tails(N):
    """Configurations whose intensities fall off geometrically (what an untrained proposal draws): the tail
    sums r_k span many decades, and the density must still follow the FP64 oracle."""
    S, R, nT, ncold = 1, 4, 2, 1
    pt = pkg.PT([N] * S, _couplings([N] * S), workload.geometric_ladder(0.5, 1.5, nT), R, 5, precision="fp32")
    pt.learn_init(n_cold=ncold, batch=128, data_per_sample=128, seed=1)
    sh = pt.learn_shape()
    rng = np.random.default_rng(N)
    rows = 64
    ratio = rng.uniform(0.3, 0.7, rows)
    s = ratio[:, None] ** np.arange(N)[None, :] * rng.uniform(0.5, 1.5, (rows, N))
    s /= s.sum(1, keepdims=True)
    a = ((N * s) ** 0.25 * np.exp(1j * rng.uniform(0, 2 * np.pi, (rows, N))))[None]
    cond = np.zeros((S, rows), np.int32)
    P = pt.learn_params().astype(np.float64)
    lq, ex, _ = pt.learn_eval(a, cond)
    lq_o, ex_o = ol.logq(P[0], a[0], cond[0], N, sh["H"], ncold, 8, emulate_bf16=True)
    assert np.allclose(ex[0], ex_o, rtol=1e-5, atol=1e-3), np.abs(ex[0] - ex_o).max()
    assert np.allclose(lq[0], lq_o, rtol=1e-4, atol=2e-3), np.abs(lq[0] - lq_o).max()


@pytest.mark.parametrize("N,rows", [(16, 1), (48, 72), (64, 128)])
def test_learn_eval_single_launch_forward_matches_oracle(N, rows):
    """Without a gradient and with at most 128 rows per sample the network runs as one fused launch (three
    tcgen05 products, hidden activations in shared memory).  It must give the three-GEMM path's result bit for
    bit (same products in the same K order, same epilogue arithmetic), and follow the FP64 oracle with the
    BF16 rounding points emulated.  Against the oracle a hidden value that sits on a BF16 rounding boundary
    can round the other way (the oracle rounds its FP64 value, the kernel its FP32 one); with these sharp
    densities (|log q| ~ 1e3) one such flip moves log q by up to ~4e-5 |log q|, so 95% of the rows are held
    to the usual bound and every row to that allowance."""
    S, R, nT, ncold = 3, 4, 4, 3
    pt = pkg.PT([N] * S, _couplings([N] * S), workload.geometric_ladder(0.5, 1.5, nT), R, 5, precision="fp32")
    pt.learn_init(n_cold=ncold, batch=256, data_per_sample=256, seed=3)
    sh = pt.learn_shape()
    rng = np.random.default_rng(7 * N + rows)
    P = _randomise_outputs(pt.learn_params().astype(np.float64), sh, rng).astype(np.float32)
    pt.set_learn_params(P)
    a = _dirichlet(N, (S, rows), 0.5, rng).astype(np.complex64).astype(np.complex128)
    cond = rng.integers(0, ncold, (S, rows)).astype(np.int32)
    lq, ex, _ = pt.learn_eval(a, cond)
    if rows % 8 == 0:  # the gradient path takes whole groups of 8 rows
        lq_g, ex_g, _ = pt.learn_eval(a, cond, grad=True)  # the three-GEMM path
        assert np.array_equal(ex, ex_g) and np.array_equal(lq, lq_g)
    for s in range(S):
        lq_o, ex_o = ol.logq(P[s].astype(np.float64), a[s], cond[s], N, sh["H"], ncold, 8, emulate_bf16=True)
        err = np.abs(lq[s] - lq_o)
        scale = np.abs(lq_o).max()
        assert np.quantile(err, 0.95) <= 2e-3 + 1e-5 * scale, (np.quantile(err, 0.95), scale)
        assert err.max() <= 2e-3 + 5e-5 * scale, (err.max(), scale)


def test_many_conditions_take_the_global_bias_path():
    """More than 64 temperature conditions: the single-launch forward reads the conditional biases C1 from
    global memory instead of staging them in shared memory, and 70 proposal rows per sample exceed the
    one-launch sampler (per-block launches).  Densities against the oracle; global moves stay exact (the
    energies that chains taking a proposal carry are the oracle's)."""
    import oracle
    N, S, R, nT, ncold = 16, 1, 1, 72, 70
    temps = workload.geometric_ladder(0.5, 1.5, nT)
    J = [0.05 * j for j in _couplings([N] * S)]
    pt = pkg.PT([N] * S, J, temps, R, 9, precision="fp64")
    pt.learn_init(n_cold=ncold, batch=128, data_per_sample=128, seed=2)
    sh = pt.learn_shape()
    rng = np.random.default_rng(70)
    P = _randomise_outputs(pt.learn_params().astype(np.float64), sh, rng).astype(np.float32)
    pt.set_learn_params(P)
    rows = 100
    a = _dirichlet(N, (S, rows), 0.5, rng).astype(np.complex64).astype(np.complex128)
    cond = rng.integers(0, ncold, (S, rows)).astype(np.int32)
    lq, ex, _ = pt.learn_eval(a, cond)
    lq_o, _ = ol.logq(P[0].astype(np.float64), a[0], cond[0], N, sh["H"], ncold, 8, emulate_bf16=True)
    err = np.abs(lq[0] - lq_o)
    scale = np.abs(lq_o).max()
    assert np.quantile(err, 0.95) <= 2e-3 + 1e-5 * scale and err.max() <= 2e-3 + 5e-5 * scale, (err.max(), scale)
    pt.set_learn_params(_stick_breaking_biases(N, pt.learn_params().astype(np.float64), sh).astype(np.float32))
    pt.set_global_blocks(4, 7)
    a0, E0 = pt.state()
    for _ in range(4):
        pt.global_move()
    a1, E1 = pt.state()
    moved = np.any(a1.reshape(-1, N) != a0.reshape(-1, N), axis=1)
    assert moved.sum() >= 4, moved.sum()
    quads = oracle.enumerate_quads(N)
    for c in np.flatnonzero(moved):
        ref = oracle.energy(N, quads, J[0], a1.reshape(-1, N)[c])
        assert abs(E1[c] - ref) <= 1e-13 * np.abs(J[0]).sum(), (c, E1[c], ref)


def test_learn_eval_rejects_bad_arguments():
    S, N = 1, 16
    pt = pkg.PT([N], _couplings([N]), workload.geometric_ladder(0.5, 1.5, 2), 4, 1, precision="fp32")
    with pytest.raises(pkg.PTError):
        pt.global_move()  # not initialised
    with pytest.raises(pkg.PTError):
        pt.learn_init(n_cold=1, batch=100)  # batch not a multiple of 128
    pt.learn_init(n_cold=2, batch=128, data_per_sample=128)
    with pytest.raises(pkg.PTError):
        pt.learn_init(n_cold=2, batch=128, data_per_sample=128)  # twice
    a = _dirichlet(N, (S, 8), 0.5, np.random.default_rng(0))
    with pytest.raises(pkg.PTError):
        pt.learn_eval(a, np.full((S, 8), 2, np.int32))  # condition out of range
    with pytest.raises(pkg.PTError):
        pt.train(4)  # no data collected
    for lo, hi in ((3, 2), (0, 8), (-1, 3)):
        with pytest.raises(pkg.PTError):
            pt.set_global_blocks(lo, hi)
    pt2 = pkg.PT([24], _couplings([24]), workload.geometric_ladder(0.5, 1.5, 2), 4, 1, precision="fp32")
    with pytest.raises(pkg.PTError):
        pt2.learn_init(n_cold=1, batch=128)  # N not a multiple of 16


def _j0_learner(N, S, R, nT, ncold, prec, seed):
    import oracle
    J0 = [np.zeros(len(oracle.enumerate_quads(N)))] * S
    pt = pkg.PT([N] * S, J0, workload.geometric_ladder(0.5, 1.5, nT), R, seed, precision=prec)
    pt.learn_init(n_cold=ncold, batch=128, data_per_sample=128, seed=4)
    sh = pt.learn_shape()
    P = pt.learn_params().astype(np.float64)
    P[:, sh["oW3"]:sh["ob3"]] *= 3.0  # keep a configuration-dependent part
    pt.set_learn_params(_stick_breaking_biases(N, P, sh).astype(np.float32))
    return pt


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_global_moves_alone_reach_the_beta0_law(prec):
    """J = 0 (H = 0 at every temperature): global moves alone, started from Dirichlet(1) intensities, must
    reach the beta = 0 law of Eq. (8), <Y4> = <sum s_k^2> = 3/(N+2), not Dirichlet(1)'s 2/(N+1)."""
    N, S, R, nT, ncold = 16, 4, 64, 3, 2
    pt = _j0_learner(N, S, R, nT, ncold, prec, 21)
    pt.set_global_blocks(0, 0)
    rng = np.random.default_rng(3)
    pt.set_state(_dirichlet(N, (S * R * nT,), 1.0, rng).ravel())
    y4 = []
    steps = 60
    for i in range(steps):
        pt.global_move()
        if i >= steps // 2:
            a, E = pt.state()
            a = a.reshape(S, R, nT, N)[:, :, :ncold]
            s = np.abs(a) ** 4 / N
            y4.append((s * s).sum(-1))
            assert np.all(E == 0)
    y4 = np.array(y4)  # [step, S, R, ncold]
    o = pt.observables()
    acc, att = o["gm_acc"], o["gm_att"]
    assert np.all(att[:, :ncold] == steps * R) and np.all(att[:, ncold:] == 0)
    rate = acc[:, :ncold].sum() / att[:, :ncold].sum()
    assert rate > 0.1, rate
    m = y4.mean()
    chain_means = y4.mean(0).ravel()
    err = 2 * chain_means.std() / math.sqrt(chain_means.size)
    assert abs(m - 3 / (N + 2)) < 5 * err + 2e-3, (m, 3 / (N + 2), err)
    assert abs(m - 2 / (N + 1)) > 10 * err
    # the chains still satisfy the constraint
    a, _ = pt.state()
    assert np.allclose((np.abs(a.reshape(-1, N)) ** 4).sum(1), N, rtol=2e-5 if prec == "fp32" else 1e-12)


@pytest.mark.parametrize("prec,lo,hi", [("fp32", 7, 7), ("fp64", 2, 5), ("fp32", 1, 7)])
def test_tail_moves_reach_the_conditional_beta0_law(prec, lo, hi):
    """Tail moves keep the modes below the first resampled block.  Under the beta = 0 law the fractions
    s_k / r_m of the modes k >= m = hi N/8 (always resampled) are Dirichlet(1/2) over those N - m modes
    whatever the head, so <sum (s_k / r_m)^2> = 3/(n+2), n = N - m.  The chains start with these fractions
    drawn from Dirichlet(1) (2/(n+1)) and the head and tail mass from the beta = 0 law; the head must not move."""
    N, S, R, nT, ncold = 32, 4, 64, 3, 2
    pt = _j0_learner(N, S, R, nT, ncold, prec, 22)
    pt.set_global_blocks(lo, hi)
    m = hi * N // 8
    n = N - m
    rng = np.random.default_rng(5)
    C = S * R * nT
    s = _dirichlet(N, (C,), 0.5, rng)
    s = np.abs(s) ** 4 / N
    g = rng.exponential(size=(C, n))
    s[:, m:] = s[:, m:].sum(1, keepdims=True) * g / g.sum(1, keepdims=True)
    a0 = (N * s) ** 0.25 * np.exp(1j * rng.uniform(0, 2 * np.pi, (C, N)))
    pt.set_state(a0.ravel())
    a_start = pt.state()[0].reshape(S, R, nT, N)
    stat = []
    steps = 60
    for i in range(steps):
        pt.global_move()
        if i >= steps // 2:
            a = pt.state()[0].reshape(S, R, nT, N)[:, :, :ncold]
            f = np.abs(a[..., m:]) ** 4
            f = f / f.sum(-1, keepdims=True)
            stat.append((f * f).sum(-1))
    a_end = pt.state()[0].reshape(S, R, nT, N)
    lo_k = lo * N // 8
    # modes below the lowest first block never move; the warmer chains do not move at all
    assert np.array_equal(a_end[:, :, :, :lo_k], a_start[:, :, :, :lo_k])
    assert np.array_equal(a_end[:, :, ncold:], a_start[:, :, ncold:])
    o = pt.observables()
    rate = o["gm_acc"][:, :ncold].sum() / o["gm_att"][:, :ncold].sum()
    assert rate > 0.1, rate
    stat = np.array(stat)
    mean = stat.mean()
    cm = stat.mean(0).ravel()
    err = 2 * cm.std() / math.sqrt(cm.size)
    assert abs(mean - 3 / (n + 2)) < 5 * err + 2e-3, (mean, 3 / (n + 2), err)
    assert abs(mean - 2 / (n + 1)) > 10 * err
    tot = (np.abs(a_end.reshape(-1, N)) ** 4).sum(1)
    assert np.allclose(tot, N, rtol=2e-5 if prec == "fp32" else 1e-12)


def _block_E(pt, nblocks, sweeps):
    out = []
    for _ in range(nblocks):
        pt.reset_observables()
        pt.sweep(sweeps)
        st = pt.observables()["stat"]
        n = st[..., 0]
        E = st[..., 1] / n
        out.append(np.stack([E, st[..., 2] / n - E ** 2, st[..., 4] / n], -1))
    return np.array(out)


def _trained(N, S, R, temps, ncold, seed, steps=4000):
    pt = pkg.PT([N] * S, _couplings([N] * S), temps, R, seed, precision="fp32", swap_every=8, measure_every=4,
                resync_every=64)
    pt.sweep(2048)
    pt.learn_init(n_cold=ncold, batch=256, data_per_sample=R * ncold * 1024, seed=seed)
    pt.collect(16, 1024)
    losses = pt.train(steps, lr=1e-3)
    return pt, losses


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_accepted_global_moves_carry_the_energy_of_the_stored_state(prec):
    """Global moves alone (no sweeps in between): a chain that took a proposal must carry the FP64 energy
    (oracle) of the configuration it now holds, computed by the proposal path (pair-product table in shared
    memory); for FP32 chains that is the energy of the proposal as rounded to FP32, the configuration the
    chain stores (the energy of the unrounded proposal differs by ~1e-8 here).  Chains that took none keep
    their energy unchanged."""
    import oracle
    N, S, R, nT, ncold = 64, 2, 4, 4, 4
    J = [0.05 * j for j in _couplings([N] * S)]
    pt = pkg.PT([N] * S, J, workload.geometric_ladder(0.5, 1.5, nT), R, 31, precision=prec)
    pt.learn_init(n_cold=ncold, batch=128, data_per_sample=128, seed=4)
    sh = pt.learn_shape()
    pt.set_learn_params(_stick_breaking_biases(N, pt.learn_params().astype(np.float64), sh).astype(np.float32))
    pt.set_global_blocks(5, 7)
    a0, E0 = pt.state()
    for _ in range(12):
        pt.global_move()
    a, E = pt.state()
    moved = np.any(a.reshape(-1, N) != a0.reshape(-1, N), axis=1)
    assert moved.sum() >= 8, moved.sum()
    assert np.array_equal(E[~moved], E0[~moved])
    quads = oracle.enumerate_quads(N)
    a = a.reshape(S, R * nT, N)
    for c in np.flatnonzero(moved):
        s_, r_ = divmod(int(c), R * nT)
        ref = oracle.energy(N, quads, J[s_], a[s_, r_])
        assert abs(E[c] - ref) <= 1e-13 * np.abs(J[s_]).sum(), (c, E[c], ref)


@pytest.mark.parametrize("N,S,R,nT,ncold,blocks", [(64, 2, 4, 4, 4, (0, 7)), (32, 2, 8, 4, 3, (2, 6)),
                                                     (16, 2, 16, 4, 4, (0, 0)), (64, 16, 2, 32, 8, (0, 7))])
def test_one_launch_sampler_draws_the_per_block_proposals(N, S, R, nT, ncold, blocks):
    """The autoregressive sampling in one launch (network weights on chip, draws written into the next pass's
    input in distributed shared memory) must draw exactly the proposals of the per-block launches: the same
    random streams and arithmetic, so after a series of global moves both ensembles hold bit-identical states,
    energies and acceptance counts.  The last case has the learned-proposal benchmark's shape (16 samples x
    32 T x 2 replicas, the 8 coldest temperatures: 16 clusters of 4 blocks)."""
    temps = workload.geometric_ladder(0.5, 1.5, nT)
    J = [0.05 * j for j in _couplings([N] * S)]
    runs = []
    for one in (True, False):
        pt = pkg.PT([N] * S, J, temps, R, 77, precision="fp32")
        pt.learn_init(n_cold=ncold, batch=128, data_per_sample=128, seed=4)
        sh = pt.learn_shape()
        rng = np.random.default_rng(5)
        P = _randomise_outputs(pt.learn_params().astype(np.float64), sh, rng, scale=0.3)
        pt.set_learn_params(_stick_breaking_biases(N, P, sh).astype(np.float32))
        pt.set_global_blocks(*blocks)
        pt.set_global_sampler(one)
        for _ in range(6):
            pt.global_move()
        a, E = pt.state()
        o = pt.observables()
        runs.append((a, E, o["gm_acc"].copy(), o["gm_att"].copy()))
        pt.close()
    (a1, E1, acc1, att1), (a2, E2, acc2, att2) = runs
    assert acc1.sum() > 0 and np.array_equal(att1, att2)
    assert np.array_equal(acc1, acc2) and np.array_equal(a1, a2) and np.array_equal(E1, E2)


def test_training_lowers_the_nll_and_raises_acceptance():
    N, S, R, nT, ncold = 16, 4, 16, 8, 4
    temps = workload.geometric_ladder(0.4, 1.6, nT)
    pt = pkg.PT([N] * S, _couplings([N] * S), temps, R, 11, precision="fp32", swap_every=8)
    pt.sweep(2048)
    pt.learn_init(n_cold=ncold, batch=256, data_per_sample=R * ncold * 1024, seed=2)
    for _ in range(16):
        pt.global_move()
    o = pt.observables()
    before = o["gm_acc"][:, :ncold].sum() / o["gm_att"][:, :ncold].sum()
    assert pt.learn_shape()["ndata"] == 0
    pt.collect(16, 1024)
    assert pt.learn_shape()["ndata"] == 1024 * R * ncold
    losses = pt.train(4000, lr=1e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-50:].mean() < losses[:10].mean() - 1.0, (losses[:10].mean(), losses[-50:].mean())
    pt.reset_observables()
    for _ in range(16):
        pt.global_move()
    o = pt.observables()
    after = o["gm_acc"][:, :ncold].sum() / o["gm_att"][:, :ncold].sum()
    print(f"global-move acceptance at the {ncold} coldest T: {before:.4f} untrained -> {after:.4f} trained; "
          f"NLL {losses[:10].mean():.2f} -> {losses[-50:].mean():.2f}")
    assert after > before and after > 0.02


def test_global_moves_keep_the_thermal_averages():
    """Finite beta, trained proposal, global moves every 8 sweeps: per (sample, T) thermal averages of E,
    C_V and Y4 agree with the sweep-only chain (which the FP64 oracle pins) within block errors."""
    N, S, R, nT, ncold = 16, 4, 16, 8, 4
    temps = workload.geometric_ladder(0.4, 1.6, nT)
    pt, _ = _trained(N, S, R, temps, ncold, 13)
    ref = pkg.PT([N] * S, _couplings([N] * S), temps, R, 14, precision="fp32", swap_every=8, measure_every=4,
                 resync_every=64)
    ref.sweep(2048)
    pt.set_global_every(8)
    pt.sweep(512)
    nb, sw = 16, 512
    g = _block_E(pt, nb, sw)
    o = _block_E(ref, nb, sw)
    acc = pt.observables()
    mg, mo = g.mean(0), o.mean(0)
    se = np.sqrt(g.var(0, ddof=1) / nb + o.var(0, ddof=1) / nb) + 1e-12
    z = (mg - mo) / se
    rate = acc["gm_acc"][:, :ncold].sum() / max(acc["gm_att"][:, :ncold].sum(), 1)
    print(f"global-move acceptance {rate:.4f}; max |z| {np.abs(z).max():.2f}")
    assert rate > 0.01
    assert np.mean(np.abs(z) > 3.0) < 0.05, np.round(z, 2)
    assert np.abs(z).max() < 5.5, np.round(z, 2)


def test_gain_measurement_reports_ess_of_both_methods():
    """What the trained network gains over plain PT: effective samples/s of E at the coldest T (Sokal
    tau_int), both methods on the same ensemble; the averages must agree, the gain is reported as measured."""
    from paper_2511_13508_gb300 import gain
    N, S, R, nT = 16, 4, 8, 8
    temps = workload.geometric_ladder(0.4, 1.6, nT)
    pt = pkg.PT([N] * S, _couplings([N] * S), temps, R, 31, precision="fp32", swap_every=16)
    r = gain.measure(pt, n_cold=4, global_every=8, train_configs=R * 4 * 512, train_steps=3000, batch=256,
                     burn_in=2048, series=2048, rate_sweeps=2048)
    print({k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()})
    assert r["ess_per_s_plain"] > 0 and r["ess_per_s_learned"] > 0
    assert r["nll_last"] < r["nll_first"]
    assert max(r["acceptance_coldest"]) > 0.01
    assert abs(r["mean_E_coldest_plain"] - r["mean_E_coldest_learned"]) < 0.05 * abs(r["mean_E_coldest_plain"])
    # the gain is the ESS ratio, i.e. the ratio of autocorrelation times times the throughput ratio, with a
    # finite jackknife error; the same for q^2
    g = (r["tau_int_sweeps_plain"] / r["tau_int_sweeps_learned"]) * (r["sweeps_per_s_learned"] / r["sweeps_per_s_plain"])
    assert r["gain"] == pytest.approx(g, rel=1e-9)
    assert np.isfinite(r["gain_err"]) and r["gain_err"] > 0
    assert r["q2"]["gain"] > 0 and np.isfinite(r["q2"]["gain_err"])
    assert abs(r["q2"]["mean_plain"] - r["q2"]["mean_learned"]) < 0.25 * r["q2"]["mean_plain"]
    # a gain needs the acceptance to beat the break-even one: below it, no gain beyond the measurement error
    assert r["break_even_acceptance"] > 0
    if r["acceptance_mean"] < 0.5 * r["break_even_acceptance"]:
        assert r["gain"] < 1.0 + 3.0 * r["gain_err"], r
