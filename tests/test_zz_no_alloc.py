"""lbm_mix_step_noalloc: the allocation-free step for callers that cannot
allocate device memory, checked through the C ABI against the handle-based
lbm_mix_step on two consecutive steps.

The test itself allocates its device buffers with torch, as such a caller
would with memory it already owns; the entry point allocates nothing (its
scratch is a static device array of the library).  Kept in a file of its
own, collected last."""
import ctypes

import numpy as np
import pytest

from paper_1603_08221_gb300 import binding, workloads

pytestmark = pytest.mark.gpu

RTOL_RHO = 1e-5  # population and density tolerance of the parity tests
RTOL_U = 1e-4


def _weights(p):
    """Rest-equilibrium weights w_i alpha_si per species, FP32 as the kernel
    holds them (s = m_min / m_sigma)."""
    m_min = min(p["m_a"], p["m_b"])
    w = np.zeros((2, 9), dtype=np.float64)
    for sp, m in enumerate((p["m_a"], p["m_b"])):
        s = float(np.float32(m_min / m))
        w[sp, 0] = np.float32((9.0 - 5.0 * s) / 9.0)
        w[sp, 1:5] = np.float32(s / 9.0)
        w[sp, 5:9] = np.float32(s / 36.0)
    return w


def _to_strips(d, N, Nx):
    """[2][9][N][Nx] -> strip layout (x/32) * 576 N + j * 576 + i * 64 + 2 * (x%32) + sp."""
    S = (Nx + 31) // 32
    pad = np.zeros((2, 9, N, S * 32), dtype=d.dtype)
    pad[..., :Nx] = d
    return np.ascontiguousarray(pad.reshape(2, 9, N, S, 32).transpose(3, 2, 1, 4, 0)).ravel()


def _from_strips(flat, N, Nx):
    S = (Nx + 31) // 32
    a = flat.reshape(S, N, 9, 32, 2).transpose(4, 2, 1, 0, 3).reshape(2, 9, N, S * 32)
    return a[..., :Nx]


def test_noalloc_step_matches_handle_step_twice():
    torch = pytest.importorskip("torch")
    p = workloads.preset("heli_argon_320x16", N=16, N_x=100)
    N, Nx = 16, 100
    sim = binding.LbmMix(**p)
    sim.init()
    sim.step(40)
    F0 = sim.get_post_state_f64()
    ref_states, ref_recs, ref_prof = [], [], []
    for _ in range(2):
        sim.step(1)
        ref_states.append(sim.get_post_state_f64())
        ref_recs.append(sim.history(1)[-1])
        ref_prof.append(sim.separation()["Cl_profile"])

    # inputs in the library's storage format, built from the handle's state
    w = _weights(p)
    rho0 = F0.sum(axis=1)                        # [2][N][Nx] densities
    refrho = rho0.mean(axis=1).astype(np.float32)  # any fixed profile is allowed
    ref_f = w[:, :, None, None] * refrho.astype(np.float64)[:, None, None, :]
    d0 = (F0 - ref_f).astype(np.float32)
    colsum = np.zeros((4, Nx))
    colsum[0:2] = rho0.sum(axis=1)

    dev = torch.device("cuda")
    buf = [torch.from_numpy(_to_strips(d0, N, Nx)).to(dev),
           torch.zeros(18 * N * 32 * ((Nx + 31) // 32), dtype=torch.float32, device=dev)]
    cs = [torch.from_numpy(colsum).to(dev), torch.zeros((4, Nx), dtype=torch.float64, device=dev)]
    d_ref = torch.from_numpy(refrho.ravel()).to(dev)
    d_alpha = torch.ones(2 * Nx, dtype=torch.float32, device=dev)
    rec = torch.zeros(8, dtype=torch.float64, device=dev)
    prof = torch.zeros(Nx, dtype=torch.float64, device=dev)
    params = binding.make_params(**p)
    stream = torch.cuda.current_stream()

    for k in range(2):
        binding.lbm_mix_step_noalloc(params, buf[k % 2].data_ptr(), buf[(k + 1) % 2].data_ptr(),
                                     d_ref.data_ptr(), d_alpha.data_ptr(),
                                     cs[k % 2].data_ptr(), cs[(k + 1) % 2].data_ptr(),
                                     rec.data_ptr(), prof.data_ptr(), stream)
        torch.cuda.synchronize()
        d = _from_strips(buf[(k + 1) % 2].cpu().numpy().astype(np.float64), N, Nx)
        G = d + ref_f
        F = ref_states[k]
        for sp in range(2):
            inner = np.s_[sp, :, :, 1:-1]
            err = np.abs(G[inner] - F[inner]).max() / np.abs(F[inner]).max()
            assert err < RTOL_RHO, (k, sp, err)
        r = rec.cpu().numpy()
        rr = ref_recs[k]
        assert r[0] == 1.0
        assert abs(r[1] - rr[1]) < 1e-6 + 1e-3 * abs(rr[1])              # CL
        assert abs(r[3] / rr[3] - 1) < RTOL_U and abs(r[4] / rr[4] - 1) < RTOL_U  # mdot
        assert abs(r[6] / rr[6] - 1) < RTOL_RHO and abs(r[7] / rr[7] - 1) < RTOL_RHO
        assert np.abs(prof.cpu().numpy() - ref_prof[k]).max() < 1e-6
        c_out = cs[(k + 1) % 2].cpu().numpy()
        col_rho = ref_states[k].sum(axis=1).sum(axis=1)  # [2][Nx]
        assert np.abs(c_out[0:2, 1:-1] - col_rho[:, 1:-1]).max() \
            < RTOL_RHO * N * np.abs(refrho).max()


def test_noalloc_rejects_oversize_and_null():
    """More than 32768 columns do not fit the static scratch; missing buffers
    are refused.  Neither call reaches the GPU."""
    lib = binding.load()
    p = binding.make_params(N=8, N_x=40000)
    z = ctypes.c_void_p(0)
    # distinct non-null placeholders: the size check rejects before any use
    fake = [ctypes.c_void_p(256 * (k + 1)) for k in range(8)]
    st = lib.lbm_mix_step_noalloc(ctypes.byref(p), *fake, z)
    assert st == binding.LBM_EINVAL
    assert "32768" in binding.lbm_mix_last_error()
    p = binding.make_params(N=8, N_x=64)
    st = lib.lbm_mix_step_noalloc(ctypes.byref(p), *([z] * 8), z)
    assert st == binding.LBM_EINVAL
