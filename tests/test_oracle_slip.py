"""Single-gas Poiseuille flow with slip: pins of the diffuse-bounce-back
parameters r (Eq. R) and tau_q (Eq. taoq) of the oracle against the slip law
they exist to reproduce (Boundary conditions section: r and tau_q are chosen
so that the scheme realises the slip boundary condition; Eq. A12 gives its
coefficients A_1, A_2).

With identical species the mixture is one gas.  Between DBB walls, driven by
a small pressure ratio, its steady velocity across the channel is the
continuum Poiseuille profile under the second-order slip condition

    u_s = c_m lambda du/dn - A_2 lambda^2 d^2u/dn^2,

where c_m is the velocity slip coefficient of Eq. R (A_1 of Eq. A12 when
c_m = A_1), plus one O(dx) remainder that the discrete DBB scheme with
pressure ends leaves.  That remainder comes from the exact discrete solution
of the x-invariant channel, which the first test derives by brute force.
"""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
VS = math.sqrt(math.pi / 6)  # varsigma


def _moment_basis():
    c2 = CX**2 + CY**2
    rows = [np.ones(9), -4 + 3 * c2, 4 - 10.5 * c2 + 4.5 * c2**2, CX, (-5 + 3 * c2) * CX,
            CY, (-5 + 3 * c2) * CY, CX**2 - CY**2, CX * CY]
    return np.array(rows, dtype=float)


SPEC = [0, 1, 4, 3, 2, 8, 7, 6, 5]  # mirror image of c_y


def _x_invariant_channel(N, tau_s, tau_q, r, G, tau_e, tau_eps, tau_d, wall="dbb"):
    """Exact steady state of the linearised single-gas D2Q9 MRT channel with
    DBB walls (Eqs. MRT, MR, bot, bot2; wall="bsr": bounce-back fraction r,
    specular reflection 1 - r) driven by a uniform pressure gradient
    G = -dp/dx, solved as one linear system.  Around the rest state the
    x-dependent part w_i rho(x) of a pressure-driven solution streams into
    w_i rho(x) + 3 w_i c_ix G, so the x-invariant remainder sees that source
    at every streaming step and at every specular reflection, which also
    moves the population by c_ix (not at the same-node rules, which map
    w_i rho(x) to itself).  Returns u_x (= j_x, rest density 1) per row."""
    M = _moment_basis()
    Minv = np.linalg.inv(M)
    S = np.diag([1, 1 / tau_e, 1 / tau_eps, 1 / tau_d, 1 / tau_q, 1 / tau_d, 1 / tau_q,
                 1 / tau_s, 1 / tau_s])
    E = np.array([[W[i] * (1 + 3 * (CX[i] * CX[k] + CY[i] * CY[k])) for k in range(9)]
                  for i in range(9)])  # linear equilibrium w_i (rho + 3 c_i . j)
    C = np.eye(9) - Minv @ S @ M @ (np.eye(9) - E)  # one collision
    n = 9 * N
    A = np.eye(n)
    b = np.zeros(n)
    for j in range(N):
        for i in range(9):
            row = 9 * j + i
            js = j - CY[i]
            if 0 <= js < N:
                A[row, 9 * js:9 * js + 9] -= C[i]
                b[row] = 3 * W[i] * CX[i] * G
            elif wall == "dbb":  # r f^eq(rho_w, u_w = 0) + (1 - r) f'_opp, same node
                o = OPP[i]
                outgoing = [k for k in range(9) if CY[k] == CY[o]]
                for k in outgoing:
                    A[row, 9 * j:9 * j + 9] -= r * W[i] * 6 * C[k]
                A[row, 9 * j:9 * j + 9] -= (1 - r) * C[o]
            else:  # r f'_opp of the node + (1 - r) f'_spec of the upstream node
                A[row, 9 * j:9 * j + 9] -= r * C[OPP[i]] + (1 - r) * C[SPEC[i]]
                b[row] = (1 - r) * 3 * W[i] * CX[i] * G
    A[-1, :] = 1.0  # the mass is free: fix it
    b[-1] = N
    f = np.linalg.solve(A, b).reshape(N, 9)
    return f @ CX


def _discrete_slip(N, tau_s, tau_q, r, G, wall="dbb"):
    """Closed form of the exact discrete steady profile: parabolic with
    curvature G/(2 nu), nu = (tau_s - 1/2)/3, and wall value
    a = (G/nu) [H t q/2 + (16 Lambda - 3)/24 - t q/6], t = tau_s - 1/2,
    Lambda = t (tau_q - 1/2), q = r/(2 - r), H = N (DBB), or
    a = (G/nu) [H t q/2 + (16 Lambda - 3)/24], q = (1 - r)/r (BSR)."""
    t = tau_s - 0.5
    nu = t / 3
    q = r / (2 - r) if wall == "dbb" else (1 - r) / r
    lam = t * (tau_q - 0.5)
    y = np.arange(N) + 0.5
    rem = t * q / 6 if wall == "dbb" else 0.0
    a = G / nu * (N * t * q / 2 + (16 * lam - 3) / 24 - rem)
    return a + G / (2 * nu) * y * (N - y)


@pytest.mark.parametrize("wall", ["dbb", "bsr"])
def test_discrete_slip_closed_form_against_direct_solve(wall):
    """Brute force on small channels: for random relaxation times, wall
    parameters and widths the direct solve equals the closed form to
    round-off.  tau_e, tau_eps, tau_d do not enter.  DBB: with
    r/(2 - r) = varsigma c_m (Eq. R) the first term is the first-order slip
    c_m lambda du/dn (lambda = varsigma t, Eq. EQFrb); with tau_q of Eq. taoq
    at uniform tau_s the middle term is A_2 lambda^2 G/nu (the second-order
    slip) and the last, -varsigma c_m G/2, is a remainder.  BSR with
    (1 - r)/r = varsigma c_m realises both terms with no remainder: Eq.
    taoq is exact for it."""
    rng = np.random.default_rng(7)
    G = 1e-3
    for _ in range(12):
        N = int(rng.integers(4, 14))
        ts, tq = 0.55 + rng.uniform(0, 4, size=2)
        r = rng.uniform(0.0, 1.9) if wall == "dbb" else rng.uniform(0.05, 1.0)
        u = _x_invariant_channel(N, ts, tq, r, G, *rng.uniform(0.6, 2.0, size=3), wall=wall)
        ref = _discrete_slip(N, ts, tq, r, G, wall=wall)
        assert np.abs(u - ref).max() < 1e-10 * np.abs(ref).max()


def _steady(orc, N, Kn, alpha, c_m0, psi_off, L_over_H=6.0, theta=1.001, tol=1e-12,
            wall=0):
    p = dict(m_a=2.0, m_b=2.0, C_l=0.4, theta=theta, Kn_out=Kn, N=N, L_over_H=L_over_H,
             accommodation=alpha, c_m0=c_m0, psi_off=psi_off, wall=wall)
    o = orc.Oracle(p)
    o.init()
    prev = None
    xm = o.N_x // 2
    for _ in range(400):
        o.step(500)
        m = o.moments()
        rho = m["rho_a"] + m["rho_b"]
        u = (m["rho_a"] * m["ua_x"] + m["rho_b"] * m["ub_x"]) / rho
        if prev is not None and np.abs(u[:, xm] - prev).max() <= tol * np.abs(u[:, xm]).max():
            break
        prev = u[:, xm].copy()
    # masses equal m_min: number density n = rho, pressure n k_B T = n/3
    p_col = rho.mean(axis=0) / 3.0
    G = -(p_col[xm + 1] - p_col[xm - 1]) / 2.0
    lam = Kn * N * (1.0 / 3.0) / p_col[xm]  # lambda = (mu/p) sqrt(pi k_B T/(2m)), mu fixed
    mu = Kn * N * (1.0 / 3.0) * math.sqrt(6.0 / math.pi)  # by lambda_out = Kn_out H at p_out
    return u[:, xm], G, lam, mu, rho[:, xm].mean()


def _A(alpha):
    A1 = (2 - alpha) / alpha * (1 - 0.1817 * alpha)
    return A1, 1 / math.pi + A1 * A1 / 2


@pytest.mark.parametrize("N,Kn,alpha,c_m0", [
    (8, 0.05, 1.0, 1 - 0.1817),        # c_m = A_1: the textbook second-order law
    (16, 0.3, 0.8, 1 - 0.1817 * 0.8),  # c_m = A_1 at partial accommodation
    (12, 0.1, 0.6, 1.016),             # c_m != A_1
])
def test_single_gas_poiseuille_slip_uniform_mfp(orc, N, Kn, alpha, c_m0):
    """Identical species, no wall-confinement correction (Psi = 1): the
    steady mid-channel velocity equals
        G/(2 mu) y (H - y) + c_m lambda G H/(2 mu) + A_2 lambda^2 G/mu
        - varsigma c_m G/(2 rho)
    to 1e-5 (measured 3e-7, set by the 1e-3 pressure ratio's nonlinearity).
    Every coefficient of Eq. R and of the first two terms of Eq. taoq moves
    this profile: changing any one of them by 1 % (3, 24, 16, 0.5 and
    varsigma of Eq. taoq; 0.1817 and 1/pi, 1/2 of Eq. A12; the two 2s, the
    1/3 and the k_B T of Eq. R; the (2 - alpha) of c_m) gave errors of
    1.4e-4 ... 1.9e-2."""
    u, G, lam, mu, rho = _steady(orc, N, Kn, alpha, c_m0, psi_off=1)
    A1, A2 = _A(alpha)
    c_m = c_m0 * (2 - alpha) / alpha
    H = N
    y = np.arange(N) + 0.5
    u_s = c_m * lam * G * H / (2 * mu) + A2 * lam**2 * G / mu - VS * c_m * G / (2 * rho)
    ref = G / (2 * mu) * y * (H - y) + u_s
    assert G > 0
    assert np.abs(u - ref).max() < 1e-5 * ref.max()


@pytest.mark.parametrize("N,Kn,alpha,c_m0", [
    (8, 0.05, 1.0, 1 - 0.1817),
    (16, 0.3, 0.8, 1 - 0.1817 * 0.8),
    (12, 0.1, 0.6, 1.016),
])
def test_single_gas_poiseuille_slip_bsr_wall(orc, N, Kn, alpha, c_m0):
    """The bounce-back / specular-reflection wall (the comparison scheme of
    the Method validation section) with bounce-back fraction 1/(1 + X), X
    the factor of Eq. R, and tau_q of Eq. taoq realises the second-order slip
    solution exactly (measured to 3e-7, the pressure ratio's nonlinearity):
        G/(2 mu) y (H - y) + c_m lambda G H/(2 mu) + A_2 lambda^2 G/mu."""
    u, G, lam, mu, rho = _steady(orc, N, Kn, alpha, c_m0, psi_off=1, wall=1)
    A1, A2 = _A(alpha)
    c_m = c_m0 * (2 - alpha) / alpha
    y = np.arange(N) + 0.5
    ref = G / (2 * mu) * y * (N - y) + c_m * lam * G * N / (2 * mu) + A2 * lam**2 * G / mu
    assert G > 0
    assert np.abs(u - ref).max() < 1e-5 * ref.max()


def _psi(a):
    a = np.asarray(a, dtype=float)
    pos = np.maximum(a, 1e-300)
    return np.where(a > 0, 1 + (pos - 1) * np.exp(-pos) - pos * pos * scipy.special.exp1(pos), 0.0)


def _effective_slip_error(orc, N, Kn):
    u, G, lam, mu, _ = _steady(orc, N, Kn, 1.0, 1 - 0.1817, psi_off=0, L_over_H=4.0)
    A1, A2 = _A(1.0)
    H = N
    Psi = lambda s: 0.5 * (_psi(s / lam) + _psi((H - s) / lam))  # noqa: E731
    y = np.arange(N) + 0.5
    # d/dy (mu Psi du/dy) = -G with the viscosity of the effective mean free path
    interior = np.array([scipy.integrate.quad(lambda s: G * (H / 2 - s) / (mu * Psi(s)), 0, v,
                                              limit=200, epsrel=1e-12)[0] for v in y])
    slip = (u - interior).mean()
    lam_w, mu_w = lam * Psi(0.0), mu * Psi(0.0)
    law = A1 * lam_w * G * (H / 2) / mu_w + A2 * lam_w**2 * G / mu_w
    return abs(slip - law) / law


def test_single_gas_slip_effective_mfp_converges(orc):
    """Soft: with the wall-confinement correction (Psi of the effective mean
    free path) the interior follows d/dy(mu Psi du/dy) = -G, and the wall
    slip approaches the second-order law evaluated with the wall's effective
    mean free path lambda Psi(0) and viscosity mu Psi(0) (the tilde tau_s(0)
    of Eq. taoq) as the lattice is refined: 11 % at N = 8, 1.5 % at N = 16
    (Kn_out = 0.5).  The tau'_s(0) term of Eq. taoq is an O(dx^2) correction
    that this comparison cannot resolve."""
    e8 = _effective_slip_error(orc, 8, 0.5)
    e16 = _effective_slip_error(orc, 16, 0.5)
    assert e8 < 0.15 and e16 < 0.025 and e16 < e8 / 4
