"""Complex-step reference derivatives of the two-species MRT-LBM time
integration (test infrastructure only, like the rest of ``oracle/``).

The time step of Sec. 3 is restated here in vectorised numpy on complex128
arrays, in the paper's order per step: the DBB parameter r from the
reflected post-collision state (Eq. R), the density-correction factors of
the ghost columns (Eq. rho2), streaming f_i(x) = f'_i(x - c_i) with the
ghost columns of Eq. rho1 and the diffuse bounce-back of Eqs. bot, bot2,
then moments (Eq. rhou), the effective relaxation times (Eqs. EQFrb,
EQFrsp, psi, taos, taoq, A12) and the MRT collision (Eqs. MR, m, S, feq).
It uses the readings of the C oracle in this package and shares no code
with it or with the CUDA library.

Every operation is analytic in the inputs (comparisons and the minimum
over columns act on real parts), so a parameter perturbed by i h with
h = 1e-30 gives J(p + i h) = J(p) + i h J'(p) + O(h^2): the real part is
the plain FP64 forward result, and Im(J)/h the exact derivative along the
perturbation, free of the cancellation that limits finite differences.
"""
from __future__ import annotations

import numpy as np
from scipy.special import exp1

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)

# moment matrix of Eq. m (rows rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy)
M = np.array([
    [1, 1, 1, 1, 1, 1, 1, 1, 1],
    [-4, -1, -1, -1, -1, 2, 2, 2, 2],
    [4, -2, -2, -2, -2, 1, 1, 1, 1],
    [0, 1, 0, -1, 0, 1, -1, -1, 1],
    [0, -2, 0, 2, 0, 1, -1, -1, 1],
    [0, 0, 1, 0, -1, 1, 1, -1, -1],
    [0, 0, -2, 0, 2, 1, 1, -1, -1],
    [0, 1, -1, 1, -1, 0, 0, 0, 0],
    [0, 0, 0, 0, 0, 1, -1, 1, -1]], dtype=float)
MINV = np.linalg.inv(M)

DEFAULTS = dict(C_l_out=-1.0, accommodation=1.0, c_m0=1.016, tau_e=1.1, tau_eps=1.2,
                mu_ratio_a=1.0, mu_ratio_b=1.0)


def psi(a):
    """Eq. psi: psi(a) = 1 + (a - 1) e^{-a} - a^2 E_1(a), E_1 the exponential
    integral (complex arguments allowed)."""
    return 1.0 + (a - 1.0) * np.exp(-a) - a * a * exp1(a)


def dpsi(a):
    """psi'(a) = 2 e^{-a} - 2 a E_1(a)."""
    return 2.0 * np.exp(-a) - 2.0 * a * exp1(a)


def run(params: dict, steps: int, alpha=None, d_theta=0.0, d_kn=0.0, d_alpha=None,
        h: float = 1e-30):
    """Runs `steps` steps from the initial state of Sec. 2 (pressure and
    composition linear between the ends, rest equilibrium) with theta,
    Kn_out and the accommodation field [2][N_x] perturbed by i h along
    (d_theta, d_kn, d_alpha).  Returns (CL, flux, dCL, dflux, state): CL as
    in Eq. CL over the updated columns, flux = the light species' x momentum
    summed over column N_x - 2, their derivatives along the perturbation,
    and the final post-collision state (real part)."""
    p = dict(DEFAULTS)
    p.update(params)
    N = int(p["N"])
    Nx = int(p["N_x"]) if "N_x" in p else int(round(N * p["L_over_H"]))
    theta = p["theta"] + 1j * h * d_theta
    kn = p["Kn_out"] + 1j * h * d_kn
    if alpha is None:
        alpha = np.full((2, Nx), p["accommodation"])
    al = np.asarray(alpha, dtype=complex).reshape(2, Nx).copy()
    if d_alpha is not None:
        al = al + 1j * h * np.asarray(d_alpha, dtype=float).reshape(2, Nx)

    # gases and lattice units (k_B T = c_s^2 m_min = 1/3, masses / m_min, n_out = 1)
    m_min = min(p["m_a"], p["m_b"])
    mh = np.array([p["m_a"], p["m_b"]]) / m_min
    s = 1.0 / mh
    light = 0 if p["m_a"] <= p["m_b"] else 1
    c_in = p["C_l"]
    c_out = p["C_l"] if p["C_l_out"] < 0 else p["C_l_out"]
    Cin = np.empty(2)
    Cout = np.empty(2)
    Cin[light], Cin[1 - light] = c_in, 1.0 - c_in
    Cout[light], Cout[1 - light] = c_out, 1.0 - c_out
    # viscosity from lambda_out = Kn_out N at the outlet state (Sec. 2)
    mx_out = float(Cout @ mh)
    mu = kn * N * (1.0 / 3.0) / np.sqrt(np.pi / (6.0 * mx_out))
    mu_s = np.array([p["mu_ratio_a"], p["mu_ratio_b"]]) * mu
    rho_in = Cin * theta * mh            # p_s,in / (s_s c_s^2)
    rho_out = Cout * mh
    cw = W[None, :] * np.array([[(9 - 5 * si) / 4] + [si] * 8 for si in s])  # w_i alpha_si
    om_e, om_eps = 1.0 / p["tau_e"], 1.0 / p["tau_eps"]
    vs = np.sqrt(np.pi / 6.0)
    c_m = p["c_m0"] * (2.0 - al) / al                  # [2][Nx] per wall node
    A1 = (2.0 - al) / al * (1.0 - 0.1817 * al)         # Eq. A12
    A2 = 1.0 / np.pi + 0.5 * A1 * A1
    H = float(N)
    y = (np.arange(N) + 0.5)[:, None]                  # row centres, wall at j = 1/2

    # initial state: rest equilibrium of the linear profiles (Eq. feq, u = 0)
    t = np.arange(Nx) / (Nx - 1)
    n0 = theta + (1.0 - theta) * t
    C0 = Cin[:, None] + (Cout - Cin)[:, None] * t[None, :]
    rho0 = n0[None, :] * C0 * mh[:, None]              # [2][Nx]
    P = cw[:, :, None, None] * rho0[:, None, None, :] * np.ones((1, 1, N, 1))
    P = P.astype(complex)

    inner = slice(1, Nx - 1)

    def mixture(rho):
        n = s[0] * rho[0] + s[1] * rho[1]
        return n, (rho[0] + rho[1]) / n

    for _ in range(steps):
        # r of both walls from the reflected post-collision state (Eq. R, first form)
        rw = []
        for w, jw in ((0, 0), (1, N - 1)):
            n, mx = mixture(P[:, :, jw, :].sum(axis=1))
            rw.append(2.0 - 2.0 / (1.0 + c_m[w] * np.sqrt(np.pi * mx / 6.0)))
        # density correction of the ghost columns (Eq. rho2)
        rc = P.sum(axis=1).sum(axis=1)                 # [2][Nx] column sums of rho_s
        k_in = N * rho_in / (2.0 * rc[:, 1] - rc[:, 2])
        k_out = N * rho_out / (2.0 * rc[:, Nx - 2] - rc[:, Nx - 3])
        Q = P.copy()
        Q[..., 0] = k_in[:, None, None] * (2.0 * P[..., 1] - P[..., 2])
        Q[..., Nx - 1] = k_out[:, None, None] * (2.0 * P[..., Nx - 2] - P[..., Nx - 3])
        # streaming (Eq. MRT): g_i(x, j) = Q_i(x - c_x, j - c_y)
        G = np.empty_like(P)
        for i in range(9):
            G[:, i] = np.roll(Q[:, i], shift=(CY[i], CX[i]), axis=(1, 2))
        # diffuse bounce-back: unknowns from the node's own outgoing populations,
        # wall equilibrium with zero normal species flux, u_w = 0 (Eqs. bot, bot2)
        for (jw, unk, out, r) in ((0, (2, 5, 6), (4, 7, 8), rw[0]),
                                  (N - 1, (4, 7, 8), (2, 5, 6), rw[1])):
            o = P[:, list(out), jw, :]                 # [2][3][Nx]
            S_out = o.sum(axis=1)
            # rho_w s = 6 sum(outgoing): f^eq_i(rho_w) = w_i s rho_w
            for k, i in enumerate(unk):
                G[:, i, jw, :] = (1.0 - r) * o[:, k] + r * 6.0 * W[i] * S_out
        # moments (Eq. rhou, Eq. P) of the updated columns
        G = G[..., inner]
        rho = G.sum(axis=1)                            # [2][N][Nx - 2]
        jx = np.einsum("i,sijx->sjx", CX.astype(float), G)
        jy = np.einsum("i,sijx->sjx", CY.astype(float), G)
        rt = rho[0] + rho[1]
        ux = (jx[0] + jx[1]) / rt
        uy = (jy[0] + jy[1]) / rt
        n, mx = mixture(rho)
        # mean free paths (k_B T = 1/3, p = n/3, p_s = n_s / 3)
        lam = 3.0 * mu / n * np.sqrt(np.pi / (6.0 * mx))
        lam_s = [3.0 * mu_s[k] / (s[k] * rho[k]) * np.sqrt(np.pi / (6.0 * mh[k])) for k in (0, 1)]

        def Psi(l):
            return 0.5 * (psi(y / l) + psi((H - y) / l))

        tau_s = 0.5 + lam * Psi(lam) * np.sqrt(6.0 / (np.pi * mx))           # Eq. taos
        xle = [(s[k] * rho[k] / n) * lam_s[k] * Psi(lam_s[k]) for k in (0, 1)]
        br = 1.0 / np.sqrt(xle[0]) + 1.0 / np.sqrt(xle[1])
        c_td = 1.5 * np.sqrt(3.0 * (mh[0] + mh[1]) * mh[0] * mh[1])
        tau_d = 0.5 + c_td / mx * br ** -2.0                                   # Eq. EQFrsp
        # tau_q per column from the wall node of each half (Eq. taoq, with
        # tau'_s(0) = d tau~_s / dy at the wall and dx = 1)
        tq_rows = np.empty((N, Nx - 2), dtype=complex)
        half = (N + 1) // 2
        for w, jw, rows in ((0, 0, slice(0, half)), (1, N - 1, slice(half, N))):
            lw, mw = lam[jw], mx[jw]
            a = H / lw
            g_ = np.sqrt(6.0 / (np.pi * mw))
            tt = lw * 0.5 * psi(a) * g_                 # tau~_s(0) = tau_s(0) - 1/2
            dtt = 0.5 * g_ * (2.0 - dpsi(a))            # from psi'(0) = 2
            a1, a2 = A1[w, inner], A2[w, inner]
            tq = (0.5 + (3.0 + 24.0 * vs * vs * tt * tt * a2) / (16.0 * tt)
                  + dtt * (12.0 + 30.0 * tt * vs * a1) / (16.0 * tt * tt))
            tq_rows[rows] = tq[None, :]
        # MRT collision per species (Eqs. MR, m, S, feq), Omega = -M^-1 S (m - m^eq)
        u2 = ux * ux + uy * uy
        Pn = np.empty_like(G)
        for k in (0, 1):
            m = np.einsum("qi,ijx->qjx", M, G[k])
            r_ = rho[k]
            meq = np.stack([r_, r_ * (-4.0 + 2.0 * s[k] + 3.0 * u2),
                            r_ * (4.0 - 3.0 * s[k] - 3.0 * u2), r_ * ux, -r_ * ux,
                            r_ * uy, -r_ * uy, r_ * (ux * ux - uy * uy), r_ * ux * uy])
            rates = np.stack([np.zeros_like(ux), om_e + 0 * ux, om_eps + 0 * ux,
                              1.0 / tau_d, 1.0 / tq_rows, 1.0 / tau_d, 1.0 / tq_rows,
                              1.0 / tau_s, 1.0 / tau_s])
            Pn[k] = G[k] - np.einsum("iq,qjx->ijx", MINV, rates * (m - meq))
        # only the updated columns change; the end columns stay as stored
        P[..., inner] = Pn

    rc = P.sum(axis=1).sum(axis=1)                     # column sums of rho_s
    ns = s[:, None] * rc
    Cl = ns[light, inner] / (ns[0, inner] + ns[1, inner])
    k = int(np.argmin(Cl.real))
    CL = (c_in - Cl[k]) / c_in
    flux = (CX[:, None] * P[light, :, :, Nx - 2]).sum()
    return CL.real, flux.real, CL.imag / h, flux.imag / h, P.real
