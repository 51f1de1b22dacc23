"""Pins of the FP64 oracle's building blocks against facts fixed by the paper
and by mathematics: orthogonality of M (Eq. m), moments of f^eq (Eqs. feq, P),
conservation and the mid-step identity of the collision (Eqs. MR, rhou), the
BGK limit (Sec. 3.1), the exponential integral and psi (Eq. psi), and the
viscosity implied by the effective relaxation time (Eqs. EQFrb, taos)."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special

from paper_1603_08221_gb300 import workloads

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


# ----------------------------------------------------------------- Eq. (m)
def test_M_rows_are_orthogonal(orc):
    """P1: the rows of M are mutually orthogonal with the squared norms
    9, 36, 36, 6, 12, 6, 12, 4, 4 (exact integers)."""
    M = orc.matrix_M()
    G = M @ M.T
    assert np.array_equal(G, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]).astype(float))
    # first row: mass; rows 3 and 5: the velocity components of the lattice.
    assert np.array_equal(M[0], np.ones(9))
    assert np.array_equal(M[3], CX.astype(float))
    assert np.array_equal(M[5], CY.astype(float))
    # energy row is 3 c^2 - 4 (standard D2Q9 moment basis)
    assert np.array_equal(M[1], 3.0 * (CX**2 + CY**2) - 4.0)


def test_gauss_jordan_inverse_matches_transpose_form(orc):
    """P1: the oracle's Gauss-Jordan M^-1 equals M^T diag(1/|row|^2)."""
    M = orc.matrix_M()
    Minv = orc.matrix_Minv()
    closed = M.T @ np.diag(1.0 / np.array([9, 36, 36, 6, 12, 6, 12, 4, 4.0]))
    assert np.allclose(Minv, closed, rtol=0, atol=1e-15)
    assert np.allclose(Minv @ M, np.eye(9), atol=1e-14)


# ----------------------------------------------------------------- Eq. feq
@pytest.mark.parametrize("s", [1.0, 0.5, 4.003 / 39.948, 20.18 / 39.948])
def test_feq_moments(orc, s):
    """P2: sum_i w_i alpha_i = 1; f^eq carries rho_s and rho_s u; its second
    moment is p_s I + rho_s u u with p_s = n_s k_B T = rho_s s / 3 (Eq. P with
    k_B T = m_min c_s^2), and M f^eq has the closed form derived from the
    moment basis: e = rho(-4 + 2s + 3u^2), eps = rho(4 - 3s - 3u^2)."""
    assert abs(orc.feq(1.0, s, 0.0, 0.0).sum() - 1.0) < 1e-15
    rho, ux, uy = 1.7, 0.03, -0.011
    fe = orc.feq(rho, s, ux, uy)
    assert abs(fe.sum() - rho) < 1e-14
    assert abs((CX * fe).sum() - rho * ux) < 1e-15
    assert abs((CY * fe).sum() - rho * uy) < 1e-15
    p_s = rho * s / 3.0
    assert abs((CX * CX * fe).sum() - (p_s + rho * ux * ux)) < 1e-14
    assert abs((CY * CY * fe).sum() - (p_s + rho * uy * uy)) < 1e-14
    assert abs((CX * CY * fe).sum() - rho * ux * uy) < 1e-15
    u2 = ux * ux + uy * uy
    m = orc.matrix_M() @ fe
    expect = rho * np.array([1, -4 + 2 * s + 3 * u2, 4 - 3 * s - 3 * u2, ux, -ux, uy, -uy,
                             ux * ux - uy * uy, ux * uy])
    assert np.allclose(m, expect, rtol=0, atol=1e-14)
    # every rest population is positive for 0 < s <= 1
    assert (orc.feq(1.0, s, 0, 0) > 0).all()


# ----------------------------------------------------------- collision
def _rand_node(seed):
    rng = np.random.default_rng(seed)
    fa = rng.uniform(0.05, 0.15, 9)
    fb = 10.0 * rng.uniform(0.05, 0.15, 9)
    return fa, fb


def _sim(orc, **kw):
    p = workloads.preset("heli_argon_320x16")
    p.update(N=8, L_over_H=1.0)
    p.update(kw)
    return orc.Oracle(p)


def _macro(f):
    return f.sum(), (CX * f).sum(), (CY * f).sum()


@pytest.mark.parametrize("seed", range(5))
def test_collision_conserves_species_mass_and_total_momentum(orc, seed):
    """P3: rho_s is conserved per species and sum_s j_s is conserved."""
    o = _sim(orc)
    fa, fb = _rand_node(seed)
    tau = np.random.default_rng(100 + seed).uniform(0.6, 3.0, 9)
    tau[3] = tau[5]  # tau_d on both momentum rows (Eq. S)
    oa, ob = o.collide_node(fa, fb, tau)
    for f, g in ((fa, oa), (fb, ob)):
        assert abs(f.sum() - g.sum()) < 1e-13 * f.sum()
    jx0 = (CX * fa).sum() + (CX * fb).sum()
    jy0 = (CY * fa).sum() + (CY * fb).sum()
    assert abs(jx0 - (CX * oa).sum() - (CX * ob).sum()) < 1e-14
    assert abs(jy0 - (CY * oa).sum() - (CY * ob).sum()) < 1e-14


@pytest.mark.parametrize("seed", range(5))
def test_each_moment_relaxes_with_its_own_time(orc, seed):
    """Eqs. MR and S: in moment space m'_k - m^eq_k = (1 - 1/tau_k)(m_k - m^eq_k)
    with tau in the order (rho, e, eps, d, q, d, q, s, s)."""
    o = _sim(orc)
    fa, fb = _rand_node(seed)
    rng = np.random.default_rng(200 + seed)
    tau = np.array([1.0, 1.1, 1.2, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])
    td, tq, ts = rng.uniform(0.6, 3.0, 3)
    tau[3] = tau[5] = td
    tau[4] = tau[6] = tq
    tau[7] = tau[8] = ts
    oa, ob = o.collide_node(fa, fb, tau)
    M = orc.matrix_M()
    rho = fa.sum() + fb.sum()
    ux = ((CX * fa).sum() + (CX * fb).sum()) / rho
    uy = ((CY * fa).sum() + (CY * fb).sum()) / rho
    c = o.constants()
    for f, g, s in ((fa, oa, c["s_a"]), (fb, ob, c["s_b"])):
        meq = M @ orc.feq(f.sum(), s, ux, uy)
        lhs = M @ g - meq
        rhs = (1.0 - 1.0 / tau) * (M @ f - meq)
        assert np.allclose(lhs, rhs, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_mid_step_species_momentum(orc, seed):
    """P11: the species momentum of Eq. rhou equals the mean of the pre- and
    post-collision momenta: rho_s u_s = (j_s + j'_s)/2."""
    o = _sim(orc)
    fa, fb = _rand_node(seed)
    td = np.random.default_rng(300 + seed).uniform(0.6, 3.0)
    tau = np.array([1.0, 1.1, 1.2, td, 1.3, td, 1.3, 0.9, 0.9])
    oa, ob = o.collide_node(fa, fb, tau)
    rho = fa.sum() + fb.sum()
    u = np.array([(CX * (fa + fb)).sum(), (CY * (fa + fb)).sum()]) / rho
    for f, g in ((fa, oa), (fb, ob)):
        j = np.array([(CX * f).sum(), (CY * f).sum()])
        jp = np.array([(CX * g).sum(), (CY * g).sum()])
        eq_rhou = (2 * td - 1) / (2 * td) * j + f.sum() * u / (2 * td)
        assert np.allclose(0.5 * (j + jp), eq_rhou, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("masses", [(workloads.HE, workloads.AR), (workloads.AR, workloads.NE)])
def test_moments_and_separation_of_a_given_state_unequal_masses(orc, masses):
    """orc_moments and orc_separation on a random state of two gases of
    unequal mass (the light one first, then second):
      - rho_s u_s of Eq. rhou is the mean of the species momenta before and
        after one collision with the node's own tau_d (j'_s from the
        Gauss-Jordan collision, not from the weights of Eq. rhou);
      - C_l(x) of Eq. C is the column's light-species number fraction
        sum_j n_l / sum_j (n_a + n_b), n_s = rho_s / m_s, from the raw
        populations (a mass fraction would differ by the 1:10 or 1:2 mass
        ratio);
      - CL of Eq. CL uses the imposed inlet fraction; mdot_s is the mean
        over the updated columns of sum_j rho_s u_s,x."""
    m_a, m_b = masses
    N, Nx = 5, 9
    o = orc.Oracle(dict(m_a=m_a, m_b=m_b, C_l=0.4, theta=2.0, Kn_out=0.2, N=N, N_x=Nx))
    f = workloads.random_post_state(N, Nx, seed=21)
    o.set_post_state(f)
    mom = o.moments()
    sep = o.separation()
    light = 0 if m_a < m_b else 1
    mass = (m_a, m_b)
    jbar = np.zeros((2, N, Nx))
    for x in range(1, Nx - 1):
        for j in range(N):
            fa, fb = f[0, :, j, x], f[1, :, j, x]
            t = o.node_taus(fa, fb, j)
            tau = np.array([1.0, 1.1, 1.2, t["tau_d"], 1.3, t["tau_d"], 1.3, t["tau_s"],
                            t["tau_s"]])
            oa, ob = o.collide_node(fa, fb, tau)
            for sp, (pre, post) in enumerate(((fa, oa), (fb, ob))):
                jx = 0.5 * ((CX * pre).sum() + (CX * post).sum())
                jy = 0.5 * ((CY * pre).sum() + (CY * post).sum())
                rho = pre.sum()
                key = "ua" if sp == 0 else "ub"
                assert abs(mom[key + "_x"][j, x] * rho - jx) < 1e-13 * rho
                assert abs(mom[key + "_y"][j, x] * rho - jy) < 1e-13 * rho
                jbar[sp, j, x] = jx
    n = f.sum(axis=1) / np.array(mass)[:, None, None]  # number densities [2][N][Nx]
    C = n[light].sum(axis=0) / n.sum(axis=(0, 1))
    inner = slice(1, Nx - 1)
    assert np.allclose(sep["Cl_profile"][inner], C[inner], rtol=1e-14, atol=0)
    assert sep["Cl_profile"][0] == 0.4 and sep["Cl_profile"][-1] == 0.4
    xm = 1 + int(np.argmin(C[inner]))
    assert sep["x_min"] == xm
    assert abs(sep["CL"] - (0.4 - C[xm]) / 0.4) < 1e-14
    for sp, key in ((0, "mdot_a"), (1, "mdot_b")):
        expect = jbar[sp][:, inner].sum(axis=0).mean()
        assert abs(sep[key] - expect) < 1e-13 * abs(expect)


@pytest.mark.parametrize("tau", [0.7, 1.0, 1.9])
def test_bgk_limit(orc, tau):
    """P12: with all relaxation times equal, the MRT collision is the BGK
    collision f' = f - (f - f^eq)/tau (Sec. 3.1)."""
    o = _sim(orc)
    fa, fb = _rand_node(7)
    oa, ob = o.collide_node(fa, fb, np.full(9, tau))
    rho = fa.sum() + fb.sum()
    ux = (CX * (fa + fb)).sum() / rho
    uy = (CY * (fa + fb)).sum() / rho
    c = o.constants()
    for f, g, s in ((fa, oa, c["s_a"]), (fb, ob, c["s_b"])):
        bgk = f - (f - orc.feq(f.sum(), s, ux, uy)) / tau
        assert np.allclose(g, bgk, rtol=1e-13, atol=1e-15)


# ----------------------------------------------------- special functions
XS = np.concatenate([np.geomspace(1e-6, 0.99, 25), [1.0], np.geomspace(1.01, 600, 40)])


def test_E1_matches_scipy(orc):
    """P9: the oracle's E_i (series / continued fraction) equals E_1 to a few
    units in the last place (the continued fraction loses ~5e-15 near x = 1)."""
    for x in XS:
        ref = scipy.special.exp1(x)
        assert abs(orc.E1(x) - ref) <= 1e-14 * ref + 1e-300, x


@pytest.mark.parametrize("x", [0.05, 0.5, 1.0, 2.0, 7.5])
def test_E1_matches_quadrature_of_definition(orc, x):
    """P9: E_i(x) = int_1^inf t^-1 e^{-xt} dt (below Eq. psi)."""
    val, err = scipy.integrate.quad(lambda t: math.exp(-x * t) / t, 1.0, np.inf,
                                    epsabs=0, epsrel=1e-13, limit=200)
    assert abs(orc.E1(x) - val) < 1e-12 * val


def test_E1_branches_join(orc):
    lo = orc.E1(1.0 - 1e-12)
    hi = orc.E1(1.0 + 1e-12)
    assert abs(lo - hi) < 1e-12


def test_psi_limits_and_derivative(orc):
    """P9: psi(0) = 0, psi -> 1 for large alpha, psi'(0) = 2 and psi is
    increasing; the closed-form derivative matches central differences."""
    assert orc.psi(0.0) == 0.0
    assert abs(orc.psi(60.0) - 1.0) < 1e-15
    h = 1e-7
    assert abs(orc.psi(h) / h - 2.0) < 1e-5
    a = np.geomspace(1e-3, 20, 200)
    v = np.array([orc.psi(t) for t in a])
    assert (np.diff(v) > 0).all() and (v > 0).all() and (v < 1).all()
    for t in [0.01, 0.3, 1.0, 3.0, 9.0]:
        hh = 1e-5 * max(t, 1e-2)
        fd = (orc.psi(t + hh) - orc.psi(t - hh)) / (2 * hh)
        assert abs(fd - orc.dpsi(t)) < 1e-8


def test_Psi_symmetry_and_wall_value(orc):
    """P9: Psi(y) = Psi(H - y); Psi(0) = psi(H/lambda)/2; Psi -> 1 in the
    middle of a wide channel."""
    H = 16.0
    for lam in [0.3, 1.6, 5.0, 40.0]:
        for y in [0.5, 3.5, 7.9]:
            assert abs(orc.Psi(y, H, lam) - orc.Psi(H - y, H, lam)) < 1e-15
        assert abs(orc.Psi(0.0, H, lam) - 0.5 * orc.psi(H / lam)) < 1e-16
    assert abs(orc.Psi(5000.0, 10000.0, 1.0) - 1.0) < 1e-15


@pytest.mark.parametrize("lam,mx", [(0.8, 5.49), (3.0, 1.0), (25.6, 1.6)])
def test_wall_derivative_of_tau_s(orc, lam, mx):
    """P10: tau'_s(0) used in Eq. taoq equals the one-sided finite-difference
    slope of tilde tau_s(y) = lambda Psi(y) sqrt(6/(pi m_x)) at the wall.
    psi'' has a log singularity at 0, so the second-order one-sided stencil
    is checked at the h ln h accuracy it can reach."""
    H = 16.0
    g = math.sqrt(6 / (math.pi * mx))
    closed = 0.5 * g * (orc.dpsi(0.0) - orc.dpsi(H / lam))
    for h in [1e-4, 1e-5]:
        f0, f1, f2 = (orc.tau_s_tilde(k * h, H, lam, mx) for k in range(3))
        fd = (-3 * f0 + 4 * f1 - f2) / (2 * h)
        assert abs(fd - closed) < 5 * h / lam * abs(math.log(h / lam)) + 1e-9


# ------------------------------------------------- relaxation-time pins
def _bulk_sim(orc, **kw):
    p = dict(m_a=20.18, m_b=39.948, C_l=0.3, theta=2.0, Kn_out=0.001, N=4000, N_x=4)
    p.update(kw)
    return orc.Oracle(p)


@pytest.mark.parametrize("seed", range(4))
def test_tau_s_gives_the_imposed_viscosity(orc, seed):
    """Eqs. EQFrb, taos with lambda = (mu/p) sqrt(pi k_B T/(2 m_x)): the LBE
    shear viscosity rho c_s^2 (tau_s - 1/2) equals mu times the wall factor
    Psi(y), i.e. mu itself wherever Psi = 1."""
    o = _bulk_sim(orc)
    fa, fb = _rand_node(seed)
    c = o.constants()
    rho = fa.sum() + fb.sum()
    for j in [0, 3, 1999]:
        t = o.node_taus(fa, fb, j)
        Psi = orc.Psi(j + 0.5, 4000.0, t["lam"])
        assert abs(rho * (t["tau_s"] - 0.5) / 3.0 - c["mu"] * Psi) < 1e-12 * c["mu"]
    t = o.node_taus(fa, fb, 1999)
    assert abs(rho * (t["tau_s"] - 0.5) / 3.0 - c["mu"]) < 1e-12 * c["mu"]


def test_mu_reproduces_outlet_knudsen(orc):
    """Kn_out = lambda_out / H (Sec. 2): at the outlet state the mixture mean
    free path from mu is Kn_out * N."""
    for name in ["heli_argon_320x16", "neon_argon_2048x32"]:
        p = workloads.preset(name)
        o = orc.Oracle(dict(p, N_x=8))
        c = o.constants()
        C = p["C_l"]
        fa = orc.feq(c["rho_out_a"], c["s_a"], 0, 0)
        fb = orc.feq(c["rho_out_b"], c["s_b"], 0, 0)
        t = o.node_taus(fa, fb, 0)
        assert abs(t["lam"] - p["Kn_out"] * p["N"]) < 1e-12 * t["lam"]
        # the outlet number density is 1 and its light fraction is C_l
        n_a = c["rho_out_a"] * c["s_a"]
        n_b = c["rho_out_b"] * c["s_b"]
        assert abs(n_a + n_b - 1.0) < 1e-14
        assert abs(n_a - C) < 1e-14  # species a is the light one here


def test_tau_d_identical_species_bulk_closed_form(orc):
    """Eq. EQFrsp for m_a = m_b and mu_a = mu_b = mu in the bulk (Psi = 1):
    x_s lambda_s = (mu/p) sqrt(pi/6) for both species, so
    tau_d - 1/2 = (3/2) sqrt(6) (mu/p) sqrt(pi/6) / 4 and, with
    tau_s - 1/2 = 3 mu / rho, (tau_d - 1/2)/(tau_s - 1/2) = 3 sqrt(pi) / 8."""
    o = _bulk_sim(orc, m_a=1.0, m_b=1.0)
    for seed in range(3):
        fa, fb = _rand_node(seed)
        fb = fb / 10.0
        t = o.node_taus(fa, fb, 1999)
        ratio = (t["tau_d"] - 0.5) / (t["tau_s"] - 0.5)
        assert abs(ratio - 3 * math.sqrt(math.pi) / 8) < 1e-12


def test_tau_d_symmetric_in_species(orc):
    """Eq. EQFrsp is symmetric under exchanging the species labels."""
    fa, fb = _rand_node(3)
    o1 = _bulk_sim(orc, m_a=4.003, m_b=39.948, mu_ratio_a=0.8, mu_ratio_b=1.3)
    o2 = _bulk_sim(orc, m_a=39.948, m_b=4.003, mu_ratio_a=1.3, mu_ratio_b=0.8, C_l=0.3)
    for j in [0, 5, 1999]:
        t1 = o1.node_taus(fa, fb, j)
        t2 = o2.node_taus(fb, fa, j)
        assert abs(t1["tau_d"] - t2["tau_d"]) < 1e-13 * t1["tau_d"]
        assert abs(t1["tau_s"] - t2["tau_s"]) < 1e-13 * t1["tau_s"]


def test_tau_d_scales_with_mean_free_path_in_bulk(orc):
    """In the bulk, tau_d - 1/2 is proportional to the species mean free paths
    ([1/sqrt(x lambda) + ...]^-2 is homogeneous of degree one): scaling all
    viscosities by k scales tau_d - 1/2 and tau_s - 1/2 by k."""
    fa, fb = _rand_node(4)
    o1 = _bulk_sim(orc, Kn_out=0.001)
    o2 = _bulk_sim(orc, Kn_out=0.003)
    t1 = o1.node_taus(fa, fb, 1999)
    t2 = o2.node_taus(fa, fb, 1999)
    assert abs((t2["tau_d"] - 0.5) / (t1["tau_d"] - 0.5) - 3.0) < 1e-11
    assert abs((t2["tau_s"] - 0.5) / (t1["tau_s"] - 0.5) - 3.0) < 1e-11


def test_dbb_r_forms_agree_for_identical_species(orc):
    """Eq. R prints two forms; with m_sigma = m_x = m_min (identical species)
    both give 2 - 2 / (1 + c_m sqrt(pi/6)).  r = 0 without slip (c_m = 0)
    and r = 1 when c_m sqrt(pi m_x/6) = 1."""
    cm = 1.016
    assert abs(orc.dbb_r(cm, 1.0, 1.0) - (2 - 2 / (1 + cm * math.sqrt(math.pi / 6)))) < 1e-15
    assert orc.dbb_r(0.0, 1.0, 3.0) == 0.0
    mx = 6 / (math.pi * cm * cm)
    assert abs(orc.dbb_r(cm, 1.0, mx) - 1.0) < 1e-14
