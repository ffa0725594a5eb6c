"""FP64 oracle of the learned global-move proposal (test infrastructure only; the product never imports it).

Written from the definition of the proposal (the paper has none; it is an exact Metropolis-Hastings
global move added to the Parallel-Tempering path of arXiv 2511.13508, whose target is Eq. (8)):

  coordinates   s_k = |a_k|^4 / sum_i |a_i|^4 (simplex), stick breaking v_k = s_k / R_k with
                R_k = sum_{i>=k} s_i, u_k = logit(v_k) (k <= N-2); gauge-fixed phases
                phi~_k = phi_k - phi_0 - k (phi_1 - phi_0) mod 2 pi (so phi~_0 = phi~_1 = 0)
  network       block-autoregressive MLP (MADE masks over n_blocks blocks of modes), two ReLU layers,
                conditional bias C1[cond] on the first layer; outputs per mode (mu, log sigma, m, rho_raw)
  density       u_k ~ Normal(mu_k, sigma_k) pushed through the logistic, phi~_k ~ wrapped Cauchy(m_k, rho_k),
                rho = 0.98 sigmoid(rho_raw), log sigma clipped to [-7, 3]
  surface       log density on the constraint surface w.r.t. prod_k ds_k dphi_k:
                log q(x) + extra(x),  extra = -sum_{k<=N-2} log R_k + 1/2 sum_k log s_k
  MH            log A = -beta (H' - H) + [log q + extra](x) - [log q + extra](x')

Everything is float64; torch is used only for autograd (the gradient oracle).  `emulate_bf16` rounds the
weights, the input features and the hidden activations to bfloat16 at the points where the tensor-core
network stores them, so that the comparison with the GPU isolates accumulation order.
"""
from __future__ import annotations

import math

import numpy as np
import torch

RHO_MAX = 0.98
U_SCALE = 0.25


def features(a: np.ndarray):
    """a [..., N] complex -> (u [..., N], phi~ [..., N], extra [...]) in float64."""
    a = np.asarray(a, np.complex128)
    N = a.shape[-1]
    s = np.abs(a) ** 4
    s = s / s.sum(-1, keepdims=True)
    R = np.flip(np.cumsum(np.flip(s, -1), -1), -1)           # R_k = sum_{i >= k} s_i
    Rn = np.concatenate([R[..., 1:], np.zeros(R.shape[:-1] + (1,))], -1)  # R_{k+1}
    u = np.zeros_like(s)
    u[..., : N - 1] = np.log(s[..., : N - 1]) - np.log(Rn[..., : N - 1])
    ph = np.angle(a)
    k = np.arange(N)
    phit = np.mod(ph - ph[..., :1] - k * (ph[..., 1:2] - ph[..., :1]), 2 * np.pi)
    phit[..., :2] = 0.0
    extra = -np.log(R[..., : N - 1]).sum(-1) + 0.5 * np.log(s).sum(-1)
    return u, phit, extra


def configuration(u, phit, alpha, theta):
    """Inverse of `features` for a given gauge: amplitudes with sum |a|^4 = N."""
    u = np.asarray(u, np.float64)
    N = u.shape[-1]
    s = np.zeros_like(u)
    r = np.ones(u.shape[:-1])
    for k in range(N - 1):
        s[..., k] = r / (1.0 + np.exp(-u[..., k]))   # v_k R_k
        r = r / (1.0 + np.exp(u[..., k]))            # R_{k+1} = R_k (1 - v_k)
    s[..., N - 1] = r
    ph = np.asarray(phit) + np.asarray(alpha)[..., None] + np.arange(N) * np.asarray(theta)[..., None]
    return (N * s) ** 0.25 * np.exp(1j * ph)


def masks(N, H, n_blocks):
    per = N // n_blocks
    din, dout = 3 * N, 4 * N
    deg_in = (np.arange(din) // 3) // per + 1
    deg_h = np.arange(H) % n_blocks
    blk_out = (np.arange(dout) // 4) // per
    M1 = (deg_in[None, :] <= deg_h[:, None]).astype(np.float64)
    M2 = (deg_h[None, :] <= deg_h[:, None]).astype(np.float64)
    M3 = (deg_h[None, :] <= blk_out[:, None]).astype(np.float64)
    return M1, M2, M3


def layout(N, H, ncold):
    """Offsets of one sample's parameters (the layout pt_learn_shape reports)."""
    din, dout = 3 * N, 4 * N
    o = {"oW1": 0}
    o["ob1"] = o["oW1"] + H * din
    o["oC1"] = o["ob1"] + H
    o["oW2"] = o["oC1"] + ncold * H
    o["ob2"] = o["oW2"] + H * H
    o["oW3"] = o["ob2"] + H
    o["ob3"] = o["oW3"] + dout * H
    o["psize"] = (o["ob3"] + dout + 63) // 64 * 64
    return o


def _bf16(x, on):
    """Round to bfloat16 in the forward value only; the gradient passes straight through in float64."""
    if not on:
        return x
    return x + (x.detach().to(torch.bfloat16).to(torch.float64) - x.detach())


def unpack(P, N, H, ncold):
    o = layout(N, H, ncold)
    din, dout = 3 * N, 4 * N
    return dict(W1=P[o["oW1"]:o["oW1"] + H * din].reshape(H, din), b1=P[o["ob1"]:o["ob1"] + H],
                C1=P[o["oC1"]:o["oC1"] + ncold * H].reshape(ncold, H), W2=P[o["oW2"]:o["oW2"] + H * H].reshape(H, H),
                b2=P[o["ob2"]:o["ob2"] + H], W3=P[o["oW3"]:o["oW3"] + dout * H].reshape(dout, H),
                b3=P[o["ob3"]:o["ob3"] + dout])


def input_features(u, phit, N, emulate_bf16=False):
    u = torch.as_tensor(u, dtype=torch.float64)
    phit = torch.as_tensor(phit, dtype=torch.float64)
    if emulate_bf16:
        f0 = torch.clamp(u.to(torch.float32) * U_SCALE, -4.0, 4.0).to(torch.float64)
        phit = phit.to(torch.float32).to(torch.float64)
    else:
        f0 = torch.clamp(u * U_SCALE, -4.0, 4.0)
    f0 = f0.clone()
    f0[..., N - 1] = 0.0
    X = torch.stack([f0, torch.cos(phit), torch.sin(phit)], -1).reshape(*u.shape[:-1], 3 * N)
    return _bf16(X, emulate_bf16)


def forward(P, u, phit, cond, N, H, ncold, n_blocks, emulate_bf16=False):
    """Network outputs [rows, 4N] (torch float64, differentiable in P)."""
    p = unpack(P, N, H, ncold)
    M1, M2, M3 = (torch.as_tensor(m) for m in masks(N, H, n_blocks))
    X = input_features(u, phit, N, emulate_bf16)
    cond = torch.as_tensor(np.asarray(cond), dtype=torch.long)
    Z1 = X @ _bf16(p["W1"] * M1, emulate_bf16).T + p["b1"] + p["C1"][cond]
    H1 = _bf16(torch.relu(Z1), emulate_bf16)
    Z2 = H1 @ _bf16(p["W2"] * M2, emulate_bf16).T + p["b2"]
    H2 = _bf16(torch.relu(Z2), emulate_bf16)
    return H2 @ _bf16(p["W3"] * M3, emulate_bf16).T + p["b3"]


def log_terms(O, u, phit, N):
    """Network part of log q per row: logit-normal of u_k (k <= N-2) and wrapped Cauchy of phi~_k (k >= 2)."""
    u = torch.as_tensor(u, dtype=torch.float64)
    phit = torch.as_tensor(phit, dtype=torch.float64)
    O = O.reshape(*O.shape[:-1], N, 4)
    mu, ls = O[..., 0], torch.clamp(O[..., 1], -7.0, 3.0)
    z = (u - mu) / torch.exp(ls)
    lv = -0.5 * z * z - ls - 0.5 * math.log(2 * math.pi) + torch.nn.functional.softplus(-u) + \
        torch.nn.functional.softplus(u)
    rho = RHO_MAX * torch.sigmoid(O[..., 3])
    lp = torch.log1p(-rho * rho) - math.log(2 * math.pi) - torch.log(1 + rho * rho - 2 * rho * torch.cos(phit - O[..., 2]))
    return lv[..., : N - 1].sum(-1) + lp[..., 2:].sum(-1)


def logq(P, a, cond, N, H, ncold, n_blocks, emulate_bf16=False):
    """(log q network part, extra) per configuration, float64 numpy."""
    u, phit, extra = features(a)
    with torch.no_grad():
        O = forward(torch.as_tensor(P, dtype=torch.float64), u, phit, cond, N, H, ncold, n_blocks, emulate_bf16)
        lq = log_terms(O, u, phit, N).numpy()
    return lq, extra


def nll_grad(P, a, cond, N, H, ncold, n_blocks, emulate_bf16=False):
    """Gradient of mean(-log q) over the rows with respect to the flat parameters (float64)."""
    u, phit, _ = features(a)
    Pt = torch.tensor(np.asarray(P, np.float64), requires_grad=True)
    O = forward(Pt, u, phit, cond, N, H, ncold, n_blocks, emulate_bf16)
    loss = -log_terms(O, u, phit, N).mean()
    loss.backward()
    return Pt.grad.numpy(), float(loss.detach())


def sample(P, cond, N, H, ncold, n_blocks, rng):
    """Draws from q by block: (u, phi~) for every row; float64."""
    rows = len(cond)
    per = N // n_blocks
    u = np.zeros((rows, N))
    phit = np.zeros((rows, N))
    Pt = torch.as_tensor(P, dtype=torch.float64)
    for b in range(n_blocks):
        with torch.no_grad():
            O = forward(Pt, u, phit, cond, N, H, ncold, n_blocks).numpy().reshape(rows, N, 4)
        for k in range(b * per, (b + 1) * per):
            if k <= N - 2:
                ls = np.clip(O[:, k, 1], -7.0, 3.0)
                u[:, k] = O[:, k, 0] + np.exp(ls) * rng.standard_normal(rows)
            if k >= 2:
                rho = RHO_MAX / (1.0 + np.exp(-O[:, k, 3]))
                t = np.tan(np.pi * (rng.uniform(size=rows) - 0.5))
                phit[:, k] = np.mod(O[:, k, 2] + 2.0 * np.arctan((1 - rho) / (1 + rho) * t), 2 * np.pi)
    return u, phit


def log_accept(beta, H_cur, H_prop, lq_cur, extra_cur, lq_prop, extra_prop):
    """Metropolis-Hastings log ratio of the independence move (target Eq. (8) on the constraint surface)."""
    return -beta * (H_prop - H_cur) + (lq_cur + extra_cur) - (lq_prop + extra_prop)
