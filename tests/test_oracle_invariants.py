"""Whole-step pins of the FP64 oracle: exact mass conservation (periodic box
and DBB walls), the rest state as a fixed point, the identical-species
collapse onto an independently written single-gas D2Q9 MRT solver, the
extrapolation of the pressure ends (Eqs. rho1, rho2), steady-state flux
balance, and the qualitative trends the paper reports (Sec. 4)."""
import math

import numpy as np
import pytest
import scipy.special

from paper_1603_08221_gb300 import workloads

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _masses(o):
    f = o.get_state()
    return f[0].sum(), f[1].sum()


@pytest.mark.parametrize("y_periodic", [1, 0])
def test_mass_conserved_exactly(orc, y_periodic):
    """P4 (fully periodic box) and P5 (periodic in x between DBB walls): the
    total mass of each species is constant to round-off from a random
    non-negative state.  Round-off here is one ulp of the Gauss-Jordan M^-1
    column sums (~6e-17 of the mass per step, systematic while non-equilibrium
    moments persist), so the bound grows with the step count; a wrong wall or
    streaming rule loses mass at the 1e-3 level per step."""
    p = workloads.preset("heli_argon_320x16", N=8, N_x=6, x_periodic=1,
                         y_periodic=y_periodic)
    o = orc.Oracle(p)
    o.set_post_state(workloads.random_post_state(8, 6, seed=11 + y_periodic))
    m0 = o.get_post_state()
    ma0, mb0 = m0[0].sum(), m0[1].sum()
    o.step(1)
    for _ in range(5):
        o.step(400)
        ma, mb = _masses(o)
        tol = 4e-16 * o.steps
        assert abs(ma - ma0) < tol * ma0
        assert abs(mb - mb0) < tol * mb0


def test_rest_state_is_fixed_point(orc):
    """P6: uniform densities at rest, theta = 1, DBB walls and pressure ends:
    one step maps the state onto itself (all terms of the step vanish)."""
    p = workloads.preset("heli_argon_320x16", N=6, N_x=10, theta=1.0)
    o = orc.Oracle(p)
    o.init()
    f0 = o.get_state()
    o.step(200)
    f1 = o.get_state()
    assert np.abs(f1 - f0).max() < 1e-14 * np.abs(f0).max()


def test_identical_species_keep_their_ratio(orc):
    """P7(i): with m_a = m_b both species see the same relaxation, walls and
    ends, so f_a / f_b stays C/(1-C) and there is no separation."""
    p = dict(m_a=1.0, m_b=1.0, C_l=0.3, theta=2.0, Kn_out=0.2, N=6, N_x=20)
    o = orc.Oracle(p)
    o.init()
    o.step(300)
    f = o.get_state()
    assert np.abs(f[0] / f[1] - 0.3 / 0.7).max() < 1e-12
    s = o.separation()
    assert abs(s["CL"]) < 1e-12 and abs(s["Cl_tilde"]) < 1e-12
    assert np.abs(s["Cl_profile"] - 0.3).max() < 1e-12


# --------------------------------------------------------------------------
# Independent single-gas D2Q9 MRT solver (pull form, polynomial moment basis,
# numpy inverse, scipy's E_1) for P7(ii).
def _moment_basis():
    c2 = CX**2 + CY**2
    rows = [np.ones(9), -4 + 3 * c2, 4 - 10.5 * c2 + 4.5 * c2**2, CX, (-5 + 3 * c2) * CX,
            CY, (-5 + 3 * c2) * CY, CX**2 - CY**2, CX * CY]
    return np.array(rows, dtype=float)


def _psi(a):
    a = np.asarray(a, dtype=float)
    return 1 + (a - 1) * np.exp(-a) - a * a * scipy.special.exp1(a)


class SingleGas:
    """Single-species D2Q9 MRT with the effective-MFP relaxation time, DBB
    walls and extrapolation-correction ends, unit molecular mass."""

    def __init__(self, N, Nx, theta, Kn_out, c_m0=1.016, alpha=1.0, tau_e=1.1, tau_eps=1.2):
        self.N, self.Nx = N, Nx
        self.M = _moment_basis()
        self.Minv = np.linalg.inv(self.M)
        self.rho_in, self.rho_out = theta, 1.0
        p_out = 1 / 3
        lam_out = Kn_out * N
        self.mu = lam_out * p_out * math.sqrt(6 / math.pi)
        cm = c_m0 * (2 - alpha) / alpha
        self.r = 2 - 2 / (1 + cm * math.sqrt(math.pi / 6))
        self.alpha = alpha
        self.tau_e, self.tau_eps = tau_e, tau_eps
        x = np.arange(Nx)
        rho = theta + (1 - theta) * x / (Nx - 1)
        self.P = W[:, None, None] * np.broadcast_to(rho, (N, Nx))[None].copy()

    def _lam(self, rho):
        return self.mu / (rho / 3) * math.sqrt(math.pi / 6)

    def _tau_q(self, lam):
        H = self.N
        g = math.sqrt(6 / math.pi)
        tt = lam * 0.5 * _psi(H / lam) * g
        dpsi_wall = 2 * np.exp(-H / lam) - 2 * (H / lam) * scipy.special.exp1(H / lam)
        dtt = 0.5 * g * (2 - dpsi_wall)
        vs = math.sqrt(math.pi / 6)
        A1 = (2 - self.alpha) / self.alpha * (1 - 0.1817 * self.alpha)
        A2 = 1 / math.pi + A1**2 / 2
        return 0.5 + (3 + 24 * vs**2 * tt**2 * A2) / (16 * tt) + dtt * (12 + 30 * tt * vs * A1) / (16 * tt**2)

    def step(self):
        N, Nx, P = self.N, self.Nx, self.P
        Pg = P.copy()
        rho = P.sum(axis=0)
        k_in = N * self.rho_in / (2 * rho[:, 1] - rho[:, 2]).sum()
        k_out = N * self.rho_out / (2 * rho[:, Nx - 2] - rho[:, Nx - 3]).sum()
        Pg[:, :, 0] = k_in * (2 * P[:, :, 1] - P[:, :, 2])
        Pg[:, :, -1] = k_out * (2 * P[:, :, Nx - 2] - P[:, :, Nx - 3])
        S = np.empty_like(P)
        for i in range(9):
            S[i] = np.roll(np.roll(Pg[i], CY[i], axis=0), CX[i], axis=1)
        for j, unk in ((0, (2, 5, 6)), (N - 1, (4, 7, 8))):
            opp = {2: 4, 5: 7, 6: 8, 4: 2, 7: 5, 8: 6}
            out = sum(P[opp[i], j, :] for i in unk)
            rho_w = out / (W[2] + W[5] + W[6])
            for i in unk:
                S[i, j, :] = self.r * W[i] * rho_w + (1 - self.r) * P[opp[i], j, :]
        # collide the interior
        I = slice(1, Nx - 1)
        f = S[:, :, I]
        rho = f.sum(axis=0)
        ux = (CX[:, None, None] * f).sum(axis=0) / rho
        uy = (CY[:, None, None] * f).sum(axis=0) / rho
        lam = self._lam(rho)
        y = (np.arange(N) + 0.5)[:, None]
        Psi = 0.5 * (_psi(y / lam) + _psi((N - y) / lam))
        tau_s = 0.5 + lam * Psi * math.sqrt(6 / math.pi)
        tq_bot = self._tau_q(lam[0])
        tq_top = self._tau_q(lam[N - 1])
        bottom = (2 * (np.arange(N) + 1) <= N + 1)[:, None]
        tau_q = np.where(bottom, tq_bot[None, :], tq_top[None, :])
        m = np.einsum("ki,ijx->kjx", self.M, f)
        u2 = ux**2 + uy**2
        meq = np.array([rho, rho * (-2 + 3 * u2), rho * (1 - 3 * u2), rho * ux, -rho * ux,
                        rho * uy, -rho * uy, rho * (ux**2 - uy**2), rho * ux * uy])
        rate = np.array([np.ones_like(rho), np.full_like(rho, 1 / self.tau_e),
                         np.full_like(rho, 1 / self.tau_eps), np.ones_like(rho), 1 / tau_q,
                         np.ones_like(rho), 1 / tau_q, 1 / tau_s, 1 / tau_s])
        rate[0] = 0.0  # conserved: mass
        rate[3] = rate[5] = 0.0  # conserved: momentum of a single gas
        fpost = f - np.einsum("ik,kjx->ijx", self.Minv, rate * (m - meq))
        self.P = P.copy()
        self.P[:, :, I] = fpost
        self.S = S


def test_identical_species_sum_is_single_gas_mrt(orc):
    """P7(ii): for m_a = m_b the sum f_a + f_b evolves as a single gas with the
    same effective relaxation times, DBB walls and pressure ends; compared with
    an independently written pull-form solver after 60 steps."""
    N, Nx = 6, 16
    p = dict(m_a=1.0, m_b=1.0, C_l=0.4, theta=2.0, Kn_out=0.3, N=N, N_x=Nx)
    o = orc.Oracle(p)
    o.init()
    g = SingleGas(N, Nx, theta=2.0, Kn_out=0.3)
    for _ in range(60):
        g.step()
    o.step(60)
    fs = o.get_state().sum(axis=0)
    I = slice(1, Nx - 1)
    assert np.abs(fs[:, :, I] - g.S[:, :, I]).max() < 1e-12
    fp = o.get_post_state().sum(axis=0)
    assert np.abs(fp[:, :, I] - g.P[:, :, I]).max() < 1e-12


def test_pressure_ends_reproduce_linear_fields(orc):
    """P13: a post-collision state linear in x whose end columns already hold
    the imposed densities is extrapolated exactly (kappa = 1), so the
    populations entering columns 1 and N_x - 2 from the ends are f^eq at the
    inlet and outlet densities (Eqs. rho1, rho2)."""
    p = workloads.preset("heli_argon_320x16", N=5, N_x=12)
    o = orc.Oracle(p)
    o.init()  # f^eq of densities linear from rho_in (x = 0) to rho_out (x = N_x-1)
    c = o.constants()
    o.step(1)
    f = o.get_state()
    for sp, key in ((0, "a"), (1, "b")):
        fin = orc.feq(c["rho_in_" + key], c["s_" + key], 0, 0)
        fout = orc.feq(c["rho_out_" + key], c["s_" + key], 0, 0)
        assert np.abs(f[sp, 1, :, 1] - fin[1]).max() < 1e-15 * 10
        assert np.abs(f[sp, 3, :, -2] - fout[3]).max() < 1e-15 * 10
        # diagonal ones away from the walls, too
        assert np.abs(f[sp, 5, 1:, 1] - fin[5]).max() < 1e-14
        assert np.abs(f[sp, 7, :-1, -2] - fout[7]).max() < 1e-14


def test_boundary_columns_carry_imposed_composition(orc):
    """Eq. rho2: after the correction the boundary columns carry exactly
    N rho_s,in (resp. out), so their mole fraction is C_l,in (C_l,out)."""
    p = workloads.preset("heli_argon_320x16", N=6, N_x=16, C_l_out=0.4)
    o = orc.Oracle(p)
    o.init()
    o.step(50)
    m = o.moments()
    c = o.constants()
    assert abs(m["rho_a"][:, 0].sum() - 6 * c["rho_in_a"]) < 1e-12
    assert abs(m["rho_b"][:, -1].sum() - 6 * c["rho_out_b"]) < 1e-12
    s = o.separation()
    assert s["Cl_profile"][0] == 0.5 and s["Cl_profile"][-1] == 0.4


def test_steady_state_face_flux_is_uniform(orc):
    """P8: at steady state each species' mass flux through every face of the
    channel is the same (inlet flux = outlet flux).  On this 24 x 8 channel
    the fluxes agree to 1e-9 after 5000 steps (a y-staggered mode grows slowly
    afterwards on channels this narrow)."""
    p = workloads.preset("heli_argon_320x16", N=8, N_x=24, theta=1.5, Kn_out=0.2)
    o = orc.Oracle(p)
    o.init()
    o.step(5000)
    Fa, Fb = o.face_flux()
    for F in (Fa, Fb):
        assert F.mean() > 0
        assert (F.max() - F.min()) < 1e-8 * F.mean()


# ----------------------------------------------------------- paper trends
def _terminal(orc, **kw):
    p = dict(m_a=workloads.HE, m_b=workloads.AR, C_l=0.5, theta=2.0, Kn_out=0.3, N=6,
             L_over_H=4.0)
    p.update(kw)
    o = orc.Oracle(p)
    o.init()
    o.step(8000)
    return o.separation()


def test_paper_trend_mass_ratio(orc):
    """P16 (soft, Sec. 4.3): with equal end concentrations the light species
    is depleted inside the channel (C_l,min < C_l,in, CL > 0) and He-Ar
    (mass ratio 1:10) separates more than Ne-Ar (1:2)."""
    he = _terminal(orc)
    ne = _terminal(orc, m_a=workloads.NE)
    for s in (he, ne):
        assert s["CL"] > 0 and s["Cl_profile"][1:-1].min() < 0.5
        assert 1 <= s["x_min"] <= len(s["Cl_profile"]) - 2
    assert ne["CL"] < he["CL"]


_OPEN_READINGS = (
    "under every reading tried of what the paper leaves open (r_sigma of Eq. R in "
    "its two printed forms and with m_sigma for m_min; lambda_sigma with the partial "
    "or the mixture pressure) CL moves the other way, here and for every Table 1 run "
    "on the paper's 700 x 20 lattice (oracle and GPU agree), and under species "
    "viscosity ratios 0.25 ... 1 and slip coefficients c_m0 0.5 ... 2, which the paper "
    "does not give")


@pytest.mark.xfail(strict=True, reason="Sec. 4.1 / Conclusions: CL falls as theta grows; "
                   + _OPEN_READINGS)
def test_paper_trend_pressure_ratio(orc):
    """P16 (soft, Sec. 4.1 and the Conclusions): at fixed Kn_out the
    separation degree decreases as the pressure ratio grows."""
    cl = [_terminal(orc, theta=t)["CL"] for t in (2.0, 3.0, 4.0)]
    assert cl[0] > cl[1] > cl[2]


@pytest.mark.xfail(strict=True, reason="Sec. 4.2 / Conclusions: CL grows with Kn_out; "
                   + _OPEN_READINGS)
def test_paper_trend_knudsen_number(orc):
    """P16 (soft, Sec. 4.2 and the Conclusions): at fixed theta the
    separation degree increases with the outlet Knudsen number."""
    cl = [_terminal(orc, Kn_out=k)["CL"] for k in (0.3, 1.0, 3.0)]
    assert cl[0] < cl[1] < cl[2]


def test_oracle_diverges_where_the_sweep_diverges(orc):
    """Sweep instance 42 (N = 16, 160 columns, theta = 4.6, Kn_out = 0.028)
    drives the scheme unstable: relaxation times near 1/2 and a large
    pressure drop.  The FP64 oracle blows up on it too (non-finite within
    1000 steps), so a diverged sweep instance is the method's, not the
    kernel's."""
    p = workloads.sweep_instances()[42]
    o = orc.Oracle(p)
    o.init()
    o.step(1000)
    assert not np.isfinite(o.moments()["rho_a"]).all()
