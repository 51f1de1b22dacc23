"""Reverse-mode reference gradients of the two-species MRT-LBM time
integration (test infrastructure only, like the rest of ``oracle/``).

The time step of Sec. 3 is restated with plain PyTorch CPU float64 tensor
operations, in the paper's order per step (Eq. R, Eq. rho2, streaming with
Eqs. rho1, bot, bot2, then Eqs. rhou, EQFrb, EQFrsp, psi, taos, taoq, A12
and the MRT collision of Eqs. MR, m, S, feq), with the readings of the C
oracle in this package; E_1 is written out (A&S 5.1.11 series, A&S 5.1.22
continued fraction) so that autograd differentiates it.  torch.autograd
then runs the reverse sweep, one step at a time under activation
checkpointing, and returns the gradient of CL or of the light species'
outlet flux with respect to theta, Kn_out and the whole accommodation field
in one pass.  It shares no code with the C oracle, with
``complex_step.py`` or with the CUDA library.
"""
from __future__ import annotations

import numpy as np
import torch
from torch.utils.checkpoint import checkpoint

_T = torch.float64
CX = torch.tensor([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=_T)
CY = torch.tensor([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=_T)
W = torch.tensor([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, dtype=_T)
# Eq. m: rows rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy
M = torch.tensor([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],
    [-4, -1, -1, -1, -1, 2, 2, 2, 2],
    [4, -2, -2, -2, -2, 1, 1, 1, 1],
    [0, 1, 0, -1, 0, 1, -1, -1, 1],
    [0, -2, 0, 2, 0, 1, -1, -1, 1],
    [0, 0, 1, 0, -1, 1, 1, -1, -1],
    [0, 0, -2, 0, 2, 1, 1, -1, -1],
    [0, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 1, -1, 1, -1]], dtype=_T)
MINV = torch.linalg.inv(M)
EULER_GAMMA = 0.57721566490153286061
DEFAULTS = dict(C_l_out=-1.0, accommodation=1.0, c_m0=1.016, tau_e=1.1, tau_eps=1.2,
                mu_ratio_a=1.0, mu_ratio_b=1.0)


def e1(x: torch.Tensor) -> torch.Tensor:
    """Exponential integral E_1(x), x > 0: power series (A&S 5.1.11) for
    x <= 2, continued fraction (A&S 5.1.22, evaluated backwards from a fixed
    depth) for x > 2; each branch sees arguments clamped to its own range,
    so both stay finite and autograd sees no NaN."""
    xs = torch.clamp(x, max=2.0)
    t = torch.ones_like(xs)
    s = torch.zeros_like(xs)
    for k in range(1, 25):  # terms beyond k = 24 are below 1e-14 of E_1 for x <= 2
        t = t * (-xs / k)
        s = s + t / k
    ser = -EULER_GAMMA - torch.log(xs) - s
    xc = torch.clamp(x, min=2.0)
    # E_1(x) = e^{-x} / (x + 1 - 1^2/(x + 3 - 2^2/(x + 5 - ...)))
    d = torch.zeros_like(xc)
    for k in range(44, 0, -1):  # depth 44: within 1e-14 of E_1 for x >= 2
        d = (k * k) / (xc + (2 * k + 1) - d)
    cf = torch.exp(-xc) / (xc + 1.0 - d)
    return torch.where(x <= 2.0, ser, cf)


def psi(a):
    """Eq. psi: 1 + (a - 1) e^{-a} - a^2 E_1(a)."""
    return 1.0 + (a - 1.0) * torch.exp(-a) - a * a * e1(a)


def dpsi(a):
    """psi'(a) = 2 e^{-a} - 2 a E_1(a)."""
    return 2.0 * torch.exp(-a) - 2.0 * a * e1(a)


def gradient(params: dict, steps: int, alpha=None, objective: str = "CL"):
    """Runs `steps` steps from the initial state of Sec. 2 and returns
    (J, dJ/dtheta, dJ/dKn_out, dJ/dalpha [2][N_x]) for J = "CL" (Eq. CL over
    the updated columns) or "flux" (the light species' x momentum summed
    over column N_x - 2), as numpy values."""
    p = dict(DEFAULTS)
    p.update(params)
    N = int(p["N"])
    Nx = int(p["N_x"]) if "N_x" in p else int(round(N * p["L_over_H"]))
    theta = torch.tensor(float(p["theta"]), dtype=_T, requires_grad=True)
    kn = torch.tensor(float(p["Kn_out"]), dtype=_T, requires_grad=True)
    if alpha is None:
        alpha = np.full((2, Nx), p["accommodation"])
    al = torch.tensor(np.asarray(alpha, dtype=float).reshape(2, Nx), dtype=_T,
                      requires_grad=True)

    m_min = min(p["m_a"], p["m_b"])
    mh = torch.tensor([p["m_a"] / m_min, p["m_b"] / m_min], dtype=_T)
    s = 1.0 / mh
    light = 0 if p["m_a"] <= p["m_b"] else 1
    c_in = p["C_l"]
    c_out = p["C_l"] if p["C_l_out"] < 0 else p["C_l_out"]
    Cin = torch.zeros(2, dtype=_T)
    Cout = torch.zeros(2, dtype=_T)
    Cin[light], Cin[1 - light] = c_in, 1.0 - c_in
    Cout[light], Cout[1 - light] = c_out, 1.0 - c_out
    # viscosity from lambda_out = Kn_out N at the outlet (k_B T = 1/3, n_out = 1)
    mx_out = float(Cout @ mh)
    mu = kn * N * (1.0 / 3.0) / np.sqrt(np.pi / (6.0 * mx_out))
    mu_s = torch.stack([p["mu_ratio_a"] * mu, p["mu_ratio_b"] * mu])
    rho_in = Cin * mh * theta
    rho_out = Cout * mh
    alpha_i = torch.stack([(9.0 - 5.0 * s) / 4.0] + [s] * 8, dim=1)  # [2][9]
    cw = W[None, :] * alpha_i
    om_e, om_eps = 1.0 / p["tau_e"], 1.0 / p["tau_eps"]
    vs = np.sqrt(np.pi / 6.0)
    c_m = p["c_m0"] * (2.0 - al) / al
    A1 = (2.0 - al) / al * (1.0 - 0.1817 * al)
    A2 = 1.0 / np.pi + 0.5 * A1 * A1
    H = float(N)
    y = (torch.arange(N, dtype=_T) + 0.5)[:, None]
    c_td = 1.5 * torch.sqrt(3.0 * (mh[0] + mh[1]) * mh[0] * mh[1])
    half = (N + 1) // 2

    t = torch.arange(Nx, dtype=_T) / (Nx - 1)
    n0 = theta + (1.0 - theta) * t
    C0 = Cin[:, None] + (Cout - Cin)[:, None] * t[None, :]
    rho0 = n0[None, :] * C0 * mh[:, None]
    P = (cw[:, :, None, None] * rho0[:, None, None, :]).expand(2, 9, N, Nx).clone()

    def mixture(rho):
        n = s[0] * rho[0] + s[1] * rho[1]
        return n, (rho[0] + rho[1]) / n

    def step(P, theta, kn, al):
        # r of both walls (Eq. R, first form) from the reflected post-collision state
        rw = []
        for w, jw in ((0, 0), (1, N - 1)):
            _, mx = mixture(P[:, :, jw, :].sum(dim=1))
            rw.append(2.0 - 2.0 / (1.0 + c_m[w] * torch.sqrt(np.pi * mx / 6.0)))
        # ghost columns (Eqs. rho1, rho2)
        rc = P.sum(dim=(1, 2))
        k_in = N * rho_in / (2.0 * rc[:, 1] - rc[:, 2])
        k_out = N * rho_out / (2.0 * rc[:, Nx - 2] - rc[:, Nx - 3])
        g_in = k_in[:, None, None] * (2.0 * P[..., 1] - P[..., 2])
        g_out = k_out[:, None, None] * (2.0 * P[..., Nx - 2] - P[..., Nx - 3])
        Q = torch.cat([g_in[..., None], P[..., 1:Nx - 1], g_out[..., None]], dim=-1)
        # streaming g_i(x, j) = Q_i(x - c_x, j - c_y), then the DBB unknowns
        Gi = [torch.roll(Q[:, i], shifts=(int(CY[i]), int(CX[i])), dims=(1, 2))
              for i in range(9)]
        for jw, unk, out, r in ((0, (2, 5, 6), (4, 7, 8), rw[0]),
                                (N - 1, (4, 7, 8), (2, 5, 6), rw[1])):
            S_out = sum(P[:, o, jw, :] for o in out)
            for i, o in zip(unk, out):
                row = (1.0 - r) * P[:, o, jw, :] + r * 6.0 * W[i] * S_out
                Gi[i] = torch.cat([Gi[i][:, :jw], row[:, None], Gi[i][:, jw + 1:]], dim=1)
        G = torch.stack(Gi, dim=1)[..., 1:Nx - 1]
        # moments, mean free paths, relaxation times
        rho = G.sum(dim=1)
        jx = torch.einsum("i,sijx->sjx", CX, G)
        jy = torch.einsum("i,sijx->sjx", CY, G)
        rt = rho[0] + rho[1]
        ux, uy = (jx[0] + jx[1]) / rt, (jy[0] + jy[1]) / rt
        n, mx = mixture(rho)
        lam = 3.0 * mu / n * torch.sqrt(np.pi / (6.0 * mx))
        lam_s = [3.0 * mu_s[k] / (s[k] * rho[k]) * torch.sqrt(np.pi / (6.0 * mh[k])) for k in (0, 1)]

        def Psi(l):
            return 0.5 * (psi(y / l) + psi((H - y) / l))

        tau_s = 0.5 + lam * Psi(lam) * torch.sqrt(6.0 / (np.pi * mx))
        xle = [(s[k] * rho[k] / n) * lam_s[k] * Psi(lam_s[k]) for k in (0, 1)]
        br = 1.0 / torch.sqrt(xle[0]) + 1.0 / torch.sqrt(xle[1])
        tau_d = 0.5 + c_td / mx / (br * br)
        tq = []
        for w, jw in ((0, 0), (1, N - 1)):
            lw, mw = lam[jw], mx[jw]
            a = H / lw
            g_ = torch.sqrt(6.0 / (np.pi * mw))
            tt = lw * 0.5 * psi(a) * g_
            dtt = 0.5 * g_ * (2.0 - dpsi(a))
            a1, a2 = A1[w, 1:Nx - 1], A2[w, 1:Nx - 1]
            tq.append(0.5 + (3.0 + 24.0 * vs * vs * tt * tt * a2) / (16.0 * tt)
                      + dtt * (12.0 + 30.0 * tt * vs * a1) / (16.0 * tt * tt))
        tq_rows = torch.cat([tq[0][None].expand(half, -1), tq[1][None].expand(N - half, -1)])
        # MRT collision per species
        u2 = ux * ux + uy * uy
        one = torch.ones_like(ux)
        rates = torch.stack([0 * one, om_e * one, om_eps * one, 1.0 / tau_d, 1.0 / tq_rows,
                             1.0 / tau_d, 1.0 / tq_rows, 1.0 / tau_s, 1.0 / tau_s])
        out = []
        for k in (0, 1):
            m = torch.einsum("qi,ijx->qjx", M, G[k])
            r_ = rho[k]
            meq = torch.stack([r_, r_ * (-4.0 + 2.0 * s[k] + 3.0 * u2),
                               r_ * (4.0 - 3.0 * s[k] - 3.0 * u2), r_ * ux, -r_ * ux,
                               r_ * uy, -r_ * uy, r_ * (ux * ux - uy * uy), r_ * ux * uy])
            out.append(G[k] - torch.einsum("iq,qjx->ijx", MINV, rates * (m - meq)))
        Pn = torch.stack(out)
        return torch.cat([P[..., :1], Pn, P[..., Nx - 1:]], dim=-1)

    for _ in range(steps):
        P = checkpoint(step, P, theta, kn, al, use_reentrant=False)

    rc = P.sum(dim=(1, 2))
    ns = s[:, None] * rc
    Cl = ns[light, 1:Nx - 1] / (ns[0, 1:Nx - 1] + ns[1, 1:Nx - 1])
    if objective == "CL":
        kmin = int(torch.argmin(Cl.detach()))
        J = (c_in - Cl[kmin]) / c_in
    else:
        J = (CX[:, None] * P[light, :, :, Nx - 2]).sum()
    J.backward()
    return (float(J.detach()), float(theta.grad), float(kn.grad), al.grad.numpy().copy())
