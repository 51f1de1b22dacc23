"""The discrete adjoint (lbm_adj_* through the C ABI): its FP64 forward map
against the oracle, its gradients against central finite differences of
that FP64 map and of the oracle, and the torch.autograd.Function on top.

Gradients are of CL (Eq. CL) and of the light species' outlet flux after a
fixed number of steps, with respect to theta, Kn_out and the per-wall-node
accommodation field.  Tolerance: relative error 1e-4 against FP64 central
differences with step h = 1e-6, plus the differences' own rounding noise,
64 eps |J| / h (eps = 2^-52): for a component of the accommodation
gradient a thousand times smaller than the largest, that noise is the
larger term (on the 1280 x 64 channel the differences of one such component
move from 7e-4 to 2e-6 relative to the adjoint as h goes from 1e-7 to 1e-4,
as rounding noise does)."""
import numpy as np
import pytest

import oracle
from paper_1603_08221_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

H_FD = 1e-6
RTOL_GRAD = 1e-4

SMALL = dict(m_a=workloads.HE, m_b=workloads.AR, C_l=0.5, theta=2.0, Kn_out=0.2, N=8, N_x=40)
STEPS = 300
CKPT = 7  # does not divide STEPS: the last interval is short


@pytest.fixture(scope="module", autouse=True)
def _libs():
    binding.load()
    oracle.build()


def _alpha(Nx, seed=1):
    a = workloads.random_accommodation(Nx, seed).reshape(2, Nx)
    return np.minimum(a, 1.0 - 10 * H_FD)  # room for +h in every component


def _J(p, alpha, steps, obj, ckpt=CKPT):
    a = binding.LbmAdjoint(p, steps, ckpt, alpha)
    cl, fl = a.forward()
    return cl if obj == binding.LBM_ADJ_CL else fl


def _oracle_J(p, alpha, steps, obj):
    o = oracle.Oracle(p)
    o.init()
    o.set_accommodation_field(np.ascontiguousarray(alpha.ravel()))
    o.step(steps)
    if obj == binding.LBM_ADJ_CL:
        return o.separation()["CL"]
    f = o.get_post_state()
    light = 0 if p["m_a"] <= p["m_b"] else 1
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
    return float((cx[:, None] * f[light, :, :, -2]).sum())


def _rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def _close(g, fd, J):
    """|g - fd| within 1e-4 of fd plus the central difference's rounding noise."""
    return abs(g - fd) <= RTOL_GRAD * abs(fd) + 64 * np.finfo(float).eps * abs(J) / H_FD


def test_fp64_forward_matches_oracle():
    al = _alpha(SMALL["N_x"])
    a = binding.LbmAdjoint(SMALL, STEPS, CKPT, al)
    cl, fl = a.forward()
    F = a.state()
    o = oracle.Oracle(SMALL)
    o.init()
    o.set_accommodation_field(np.ascontiguousarray(al.ravel()))
    o.step(STEPS)
    Fo = o.get_post_state()
    inner = np.s_[..., 1:-1]
    assert np.abs(F[inner] - Fo[inner]).max() <= 1e-11 * np.abs(Fo[inner]).max()
    assert abs(cl - o.separation()["CL"]) < 1e-11
    assert _rel(fl, _oracle_J(SMALL, al, STEPS, binding.LBM_ADJ_FLUX)) < 1e-10


def test_fp64_forward_matches_fp32_kernel():
    p = dict(SMALL)
    a = binding.LbmAdjoint(p, STEPS, CKPT)
    a.forward()
    F = a.state()
    g = binding.LbmMix(**p)
    g.init()
    g.step(STEPS)
    G = g.get_post_state_f64()
    inner = np.s_[..., 1:-1]
    assert np.abs(G[inner] - F[inner]).max() < 1e-5 * np.abs(F[inner]).max()


@pytest.mark.parametrize("obj", [binding.LBM_ADJ_CL, binding.LBM_ADJ_FLUX])
def test_gradient_against_fd_of_the_fp64_map(obj):
    al = _alpha(SMALL["N_x"])
    a = binding.LbmAdjoint(SMALL, STEPS, CKPT, al)
    a.forward()
    g = a.gradient(obj)
    for name in ("theta", "Kn_out"):
        pp, pm = dict(SMALL), dict(SMALL)
        pp[name] += H_FD
        pm[name] -= H_FD
        fd = (_J(pp, al, STEPS, obj) - _J(pm, al, STEPS, obj)) / (2 * H_FD)
        assert _rel(g[name], fd) < RTOL_GRAD, (name, g[name], fd)
    rng = np.random.default_rng(7)
    flat = g["alpha"].ravel()
    J0 = _J(SMALL, al, STEPS, obj)
    for k in rng.choice(flat.size, 4, replace=False):
        e = np.zeros(flat.size)
        e[k] = H_FD
        fd = (_J(SMALL, al + e.reshape(al.shape), STEPS, obj)
              - _J(SMALL, al - e.reshape(al.shape), STEPS, obj)) / (2 * H_FD)
        assert _close(flat[k], fd, J0), (k, flat[k], fd)
    for _ in range(2):
        v = rng.standard_normal(flat.size)
        v /= np.abs(v).max()
        d = (H_FD * v).reshape(al.shape)
        fd = (_J(SMALL, al + d, STEPS, obj) - _J(SMALL, al - d, STEPS, obj)) / (2 * H_FD)
        assert _rel(float(flat @ v), fd) < RTOL_GRAD


@pytest.mark.parametrize("N,Nx", [(5, 5), (4, 6), (5, 7)])
@pytest.mark.parametrize("obj", [binding.LBM_ADJ_CL, binding.LBM_ADJ_FLUX])
def test_narrow_channels_against_fd_of_the_oracle(N, Nx, obj):
    """Channels so short that the ends share columns (N_x = 5: column 2 is
    the second column of both ends; N_x = 6: the ends touch) and odd row
    counts: theta, Kn_out and every accommodation component against central
    differences of the oracle."""
    p = dict(m_a=workloads.HE, m_b=workloads.AR, C_l=0.5, theta=1.5, Kn_out=0.3, N=N, N_x=Nx)
    steps = 60
    al = _alpha(Nx, seed=2)
    a = binding.LbmAdjoint(p, steps, 7, al)
    a.forward()
    g = a.gradient(obj)
    J0 = _oracle_J(p, al, steps, obj)
    for name in ("theta", "Kn_out"):
        pp, pm = dict(p), dict(p)
        pp[name] += H_FD
        pm[name] -= H_FD
        fd = (_oracle_J(pp, al, steps, obj) - _oracle_J(pm, al, steps, obj)) / (2 * H_FD)
        assert _close(g[name], fd, J0), (name, g[name], fd)
    flat = g["alpha"].ravel()
    for k in range(flat.size):
        e = np.zeros(flat.size)
        e[k] = H_FD
        e = e.reshape(al.shape)
        fd = (_oracle_J(p, al + e, steps, obj) - _oracle_J(p, al - e, steps, obj)) / (2 * H_FD)
        assert _close(flat[k], fd, J0), (k, flat[k], fd)


@pytest.mark.parametrize("obj", [binding.LBM_ADJ_CL, binding.LBM_ADJ_FLUX])
def test_gradient_against_fd_of_the_oracle(obj):
    al = _alpha(SMALL["N_x"])
    a = binding.LbmAdjoint(SMALL, STEPS, CKPT, al)
    a.forward()
    g = a.gradient(obj)
    for name in ("theta", "Kn_out"):
        pp, pm = dict(SMALL), dict(SMALL)
        pp[name] += H_FD
        pm[name] -= H_FD
        fd = (_oracle_J(pp, al, STEPS, obj) - _oracle_J(pm, al, STEPS, obj)) / (2 * H_FD)
        assert _rel(g[name], fd) < RTOL_GRAD, (name, g[name], fd)
    k = 2 * 7  # bottom wall, column 14
    e = np.zeros(al.size)
    e[k] = H_FD
    e = e.reshape(al.shape)
    fd = (_oracle_J(SMALL, al + e, STEPS, obj) - _oracle_J(SMALL, al - e, STEPS, obj)) / (2 * H_FD)
    assert _close(g["alpha"].ravel()[k], fd, _oracle_J(SMALL, al, STEPS, obj))


def test_checkpoint_interval_does_not_change_the_gradient():
    """One interval (the forward run keeps every step: nothing is replayed),
    two (the last is kept, the first replayed) or many: the same gradient,
    bit for bit."""
    al = _alpha(SMALL["N_x"])
    out = []
    for ck in (1, 7, 150, 300, 1000):
        a = binding.LbmAdjoint(SMALL, STEPS, ck, al)
        a.forward()
        out.append(a.gradient(binding.LBM_ADJ_CL))
    for g in out[1:]:
        assert g["theta"] == out[0]["theta"] and g["Kn_out"] == out[0]["Kn_out"]
        assert np.array_equal(g["alpha"], out[0]["alpha"])


@pytest.mark.parametrize("ckpt", [7, 150, 300])
def test_repeated_gradients(ckpt):
    """Gradients of both objectives after one forward run, in turn and again:
    each equals the one of a fresh handle (the interval the forward run kept
    is replayed again once a backward sweep has reused its buffers)."""
    al = _alpha(SMALL["N_x"])
    fresh = {}
    for obj in (binding.LBM_ADJ_CL, binding.LBM_ADJ_FLUX):
        a = binding.LbmAdjoint(SMALL, STEPS, ckpt, al)
        a.forward()
        fresh[obj] = a.gradient(obj)
    a = binding.LbmAdjoint(SMALL, STEPS, ckpt, al)
    a.forward()
    for obj in (binding.LBM_ADJ_CL, binding.LBM_ADJ_FLUX, binding.LBM_ADJ_CL):
        g = a.gradient(obj)
        assert g["theta"] == fresh[obj]["theta"] and g["Kn_out"] == fresh[obj]["Kn_out"]
        assert np.array_equal(g["alpha"], fresh[obj]["alpha"])


@pytest.mark.parametrize("steps,ckpt", [(300, 7), (301, 7), (300, 30), (10, 4), (300, 300),
                                        (301, 1000), (301, 151)])
def test_state_is_kept_through_the_gradient(steps, ckpt):
    """The backward sweep replays every checkpoint interval; the final state
    of the forward run must survive it, whatever the parity of the step count
    and whether the interval divides it."""
    al = _alpha(SMALL["N_x"])
    a = binding.LbmAdjoint(SMALL, steps, ckpt, al)
    a.forward()
    before = a.state()
    a.gradient(binding.LBM_ADJ_CL)
    assert np.array_equal(a.state(), before)
    o = oracle.Oracle(SMALL)
    o.init()
    o.set_accommodation_field(np.ascontiguousarray(al.ravel()))
    o.step(steps)
    Fo = o.get_post_state()
    inner = np.s_[..., 1:-1]
    assert np.abs(before[inner] - Fo[inner]).max() <= 1e-11 * np.abs(Fo[inner]).max()


def test_autograd_function():
    torch = pytest.importorskip("torch")
    from paper_1603_08221_gb300.autograd import channel_objective
    al = _alpha(SMALL["N_x"])
    theta = torch.tensor(SMALL["theta"], dtype=torch.float64, requires_grad=True)
    kn = torch.tensor(SMALL["Kn_out"], dtype=torch.float64, requires_grad=True)
    alpha = torch.tensor(al, dtype=torch.float64, requires_grad=True)
    cl = channel_objective(theta, kn, alpha, SMALL, STEPS, CKPT)
    (2.0 * cl).backward()
    a = binding.LbmAdjoint(SMALL, STEPS, CKPT, al)
    a.forward()
    g = a.gradient(binding.LBM_ADJ_CL)
    assert theta.grad.item() == 2.0 * g["theta"]
    assert kn.grad.item() == 2.0 * g["Kn_out"]
    assert np.array_equal(alpha.grad.numpy(), 2.0 * g["alpha"])


def test_helium_argon_1280x64_5000_steps():
    """The sensitivity workload: He-Ar, C_l = 0.5, theta = 2, Kn_out = 0.2,
    1280 x 64, 5000 steps, checkpoints every 70 steps, accommodation
    1 - U(0, 0.05) per wall node.  dCL/dtheta and dCL/dKn_out, and the
    outlet-flux gradient in 16 random components and 4 random directions of
    the accommodation field, against FP64 central differences."""
    p = workloads.preset("heli_argon_1280x64")
    Nx = workloads.n_x(p)
    al = _alpha(Nx)
    steps, ck = 5000, 70
    a = binding.LbmAdjoint(p, steps, ck, al)
    _, flux = a.forward()
    g = a.gradient(binding.LBM_ADJ_CL)
    for name in ("theta", "Kn_out"):
        pp, pm = dict(p), dict(p)
        pp[name] += H_FD
        pm[name] -= H_FD
        fd = (_J(pp, al, steps, 0, steps) - _J(pm, al, steps, 0, steps)) / (2 * H_FD)
        assert _rel(g[name], fd) < RTOL_GRAD, (name, g[name], fd)
    gf = a.gradient(binding.LBM_ADJ_FLUX)["alpha"].ravel()
    rng = np.random.default_rng(11)
    for k in rng.choice(gf.size, 16, replace=False):
        e = np.zeros(gf.size)
        e[k] = H_FD
        e = e.reshape(al.shape)
        fd = (_J(p, al + e, steps, 1, steps) - _J(p, al - e, steps, 1, steps)) / (2 * H_FD)
        assert _close(gf[k], fd, flux), (k, gf[k], fd)
    for _ in range(4):
        v = rng.standard_normal(gf.size)
        v /= np.abs(v).max()
        d = (H_FD * v).reshape(al.shape)
        fd = (_J(p, al + d, steps, 1, steps) - _J(p, al - d, steps, 1, steps)) / (2 * H_FD)
        assert _close(float(gf @ v), fd, flux)


@pytest.mark.parametrize("obj", [binding.LBM_ADJ_CL, binding.LBM_ADJ_FLUX])
def test_gradient_against_the_complex_step_reference(obj):
    """Against exact derivatives of the oracle-side complex-step restatement
    of the time integration (no finite-difference noise): theta, Kn_out,
    three accommodation components and two random directions, to 1e-8."""
    from oracle import complex_step as cs
    al = _alpha(SMALL["N_x"])
    a = binding.LbmAdjoint(SMALL, STEPS, CKPT, al)
    a.forward()
    g = a.gradient(obj)
    k = 0 if obj == binding.LBM_ADJ_CL else 1

    def ref(**kw):
        return cs.run(SMALL, STEPS, al, **kw)[2 + k]

    assert _rel(g["theta"], ref(d_theta=1.0)) < 1e-8
    assert _rel(g["Kn_out"], ref(d_kn=1.0)) < 1e-8
    rng = np.random.default_rng(5)
    flat = g["alpha"].ravel()
    scale = np.abs(flat).max()
    for idx in rng.choice(flat.size, 3, replace=False):
        d = np.zeros(flat.size)
        d[idx] = 1.0
        r = ref(d_alpha=d.reshape(al.shape))
        assert abs(flat[idx] - r) <= 1e-8 * abs(r) + 1e-12 * scale, (idx, flat[idx], r)
    for _ in range(2):
        v = rng.standard_normal(flat.size)
        assert _rel(float(flat @ v), ref(d_alpha=v.reshape(al.shape))) < 1e-8


@pytest.mark.parametrize("obj,name", [(binding.LBM_ADJ_CL, "CL"), (binding.LBM_ADJ_FLUX, "flux")])
def test_whole_gradient_against_the_reverse_mode_reference(obj, name):
    """The full accommodation gradient (2 x 40 values), dJ/dtheta and
    dJ/dKn_out against the oracle-side reverse-mode reference (PyTorch CPU
    autograd over a restatement of the time integration), to 1e-8."""
    pytest.importorskip("torch")
    from oracle import reference_adjoint as ra
    steps = 100
    al = _alpha(SMALL["N_x"])
    a = binding.LbmAdjoint(SMALL, steps, CKPT, al)
    a.forward()
    g = a.gradient(obj)
    J, dth, dkn, dal = ra.gradient(SMALL, steps, al, name)
    assert _rel(g["theta"], dth) < 1e-8 and _rel(g["Kn_out"], dkn) < 1e-8
    assert np.abs(g["alpha"] - dal).max() <= 1e-8 * np.abs(dal).max()
