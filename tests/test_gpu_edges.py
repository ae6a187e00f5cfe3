"""Degenerate cases of the method on the GPU, against the FP64 oracle:

  * a filled proton shell (sd, 12 protons: one proton SD) with 2 neutrons:
    H x for k = 1, 2, 4, 8 in FP64 and FP32;
  * one species empty (sd, 0 protons, 3 neutrons, 2M = 3): one-body densities
    (no proton entries, neutron trace 3) and the strength sum rule;
  * thick restart in a space smaller than one cycle's Krylov space
    (p shell, 1 proton + 1 neutron, dim 10): the run ends with the exact
    spectrum instead of failing;
  * the failure path of the kernels' bounded waits: a wait on an mbarrier
    that nothing arrives at gives up after its limit, the kernel returns,
    bs_sync_status reports BS_ETIMEOUT once, and the context still computes
    H x equal to the oracle's.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I

torch = pytest.importorskip("torch")


@pytest.mark.gpu
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_filled_proton_shell(k):
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 12, 2, 0, +1, device=0)
    o = O.Oracle(orbits, 12, 2, 0, 0).set_interaction(spe, tb)
    assert c.dim == o.dim
    x = I.random_block(o.dim, k, seed=3 + k)
    ref = o.spmv(x)
    for dt, tdt, tol in ((N.BS_F64, torch.float64, 1e-12), (N.BS_F32, torch.float32, 1e-5)):
        xd = torch.from_numpy(x).to("cuda", tdt)
        yd = torch.full_like(xd, float("nan"))
        c.apply_H(xd, yd, k, dt)
        torch.cuda.synchronize()
        y = yd.double().cpu().numpy()
        assert np.all(np.isfinite(y))
        assert np.max(np.abs(y - ref)) <= tol * np.max(np.abs(ref)), dt
    c.sync_status()


@pytest.mark.gpu
def test_densities_and_strength_with_no_protons():
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 0, 3, 3, +1, device=0)
    o = O.Oracle(orbits, 0, 3, 3, 0).set_interaction(spe, tb)
    rng = np.random.default_rng(9)
    F = rng.standard_normal((o.dim, 2))
    X = rng.standard_normal((o.dim, 2))
    ns = sum(orb.twoj + 1 for orb in orbits)
    rho = c.density(torch.from_numpy(F).cuda(), torch.from_numpy(X).cuda(), 2, ns)
    assert np.max(np.abs(rho[0])) == 0.0
    for f in range(2):
        for j in range(2):
            ref = o.density(F[:, f], X[:, j])
            assert np.max(np.abs(rho[:, :, :, f, j] - ref)) < 1e-11
            assert abs(np.trace(rho[1, :, :, f, j]) - 3.0 * F[:, f] @ X[:, j]) < 1e-9
    W0 = I.random_block(o.dim, 2, seed=10)
    E, S, rep = c.strength(torch.from_numpy(W0).cuda(), 2, N.BS_F64, 6, 12)
    assert np.allclose(S.sum(axis=1), (W0 * W0).sum(axis=0), rtol=1e-10)
    c.sync_status()


@pytest.mark.gpu
def test_thick_restart_in_a_tiny_space():
    orbits, spe, tb = I.space("p")
    c = N.make(orbits, spe, tb, 1, 1, 0, +1, device=0)
    o = O.Oracle(orbits, 1, 1, 0, 0).set_interaction(spe, tb)
    assert c.dim == 10
    ev_d = np.linalg.eigvalsh(o.dense())
    p = torch.from_numpy(I.random_block(c.dim, 2, seed=I.PIVOT_SEED)).cuda()
    # nthick > nkeep, as the thick-restart method requires
    ev, rep = c.lanczos(p, 2, N.BS_F64, 4, 3, refine=True, nthick=4, max_restarts=5, tol=1e-10)
    assert np.max(np.abs(ev - ev_d[:3])) < 1e-9, (ev, ev_d[:3])
    c.sync_status()


@pytest.mark.gpu
def test_bounded_wait_expiry_is_reported_and_the_context_stays_usable():
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 2, 2, 0, +1, device=0)
    o = O.Oracle(orbits, 2, 2, 0, 0).set_interaction(spe, tb)
    L = N.load()
    st = torch.cuda.Stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    assert L.bs_sync_status(c.h, sp) == 0
    assert L.bs_debug_wait_expiry(c.h, 0, sp) == -1               # BS_EINVAL: limit
    assert L.bs_debug_wait_expiry(c.h, (1 << 22) + 1, sp) == -1
    for _ in range(2):
        assert L.bs_debug_wait_expiry(c.h, 2000, sp) == 0
        assert L.bs_sync_status(c.h, sp) == -7                    # BS_ETIMEOUT, read and cleared
        assert b"wait" in L.bs_last_error(c.h)
        assert L.bs_sync_status(c.h, sp) == 0
    assert torch.cuda.synchronize() is None                        # no CUDA error left behind
    x = I.random_block(o.dim, 4, seed=9)
    ref = o.spmv(x)
    xd = torch.from_numpy(x).to("cuda", torch.float64)
    yd = torch.full_like(xd, float("nan"))
    c.apply_H(xd, yd, 4, N.BS_F64, st.cuda_stream)
    c.sync_status(st.cuda_stream)
    y = yd.cpu().numpy()
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
