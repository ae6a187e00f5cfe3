"""Thick-restart block Lanczos on the GPU (bs_lanczos with nthick > 0) against
the FP64 oracle's thick-restart block Lanczos (Sec. "Thick-restart Lanczos",
Sec. "Thick-restart block Lanczos").

  * FP64, sd 4p4n (dim 28,503), k = 1, 2, 4, 8: after 0, 1 and 3 restarts from
    the same pivot the Ritz values equal the oracle's (1e-8 MeV): the kept
    Ritz vectors, the arrow-shaped T and the restarted Krylov space are the
    same; the graph-captured iteration gives the same values through restarts.
  * FP64 convergence with a tolerance: refined residuals and agreement with
    the oracle's full Lanczos.
  * FP32 k = 8, 48Cr (pf 4p4n, dim 1,963,461): converged levels within 1e-4 MeV
    of full block Lanczos with a fifth of the stored blocks.
  * argument checks.
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sd44():
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    o = O.Oracle(orbits, 4, 4, 0, 0).set_interaction(spe, tb)
    return c, o


def pivot(dim, k, dtype):
    p = I.random_block(dim, k, seed=I.PIVOT_SEED)
    return p, torch.from_numpy(p).to("cuda", torch.float64 if dtype == N.BS_F64 else torch.float32)


@pytest.mark.gpu
@pytest.mark.parametrize("k,niter,nthick", [(1, 14, 4), (2, 9, 4), (4, 7, 8), (8, 5, 16)])
def test_fp64_thick_restart_equals_oracle(sd44, k, niter, nthick):
    c, o = sd44
    ph, pd = pivot(o.dim, k, N.BS_F64)
    for restarts in (0, 1, 3):
        ev_o, _ = o.block_lanczos_thick(ph, niter, nthick, restarts, nkeep=5)
        ev, rep = c.lanczos(pd, k, N.BS_F64, niter, 5, refine=False, nthick=nthick, max_restarts=restarts)
        assert rep["restarts"] == restarts
        assert rep["matvec_blocks"] == niter + restarts * (niter - nthick // k)
        assert np.max(np.abs(ev - ev_o)) < 1e-8, (restarts, ev, ev_o)
    s = torch.cuda.Stream()
    ev_g, rep_g = c.lanczos(pd, k, N.BS_F64, niter, 5, refine=False, nthick=nthick, max_restarts=3,
                            use_graph=True, stream=s.cuda_stream)
    assert rep_g["restarts"] == 3
    assert np.max(np.abs(ev_g - ev)) <= 1e-12 * np.max(np.abs(ev))
    c.sync_status()


@pytest.mark.gpu
def test_fp64_thick_restart_converges_to_tolerance(sd44):
    c, o = sd44
    ph, pd = pivot(o.dim, 4, N.BS_F64)
    ev, rep = c.lanczos(pd, 4, N.BS_F64, 8, 3, refine=True, nthick=12, max_restarts=200, tol=1e-7)
    assert 1 <= rep["restarts"] < 200
    assert rep["resid_est"] <= 1e-7
    assert max(rep["residual"][:3]) < 1e-6, rep["residual"]
    ev_l = o.lanczos(ph[:, 0], 300, nkeep=3)
    assert np.max(np.abs(ev - ev_l)) < 1e-8, (ev, ev_l)


@pytest.mark.gpu
def test_fp32_thick_restart_48cr_within_1e4_mev():
    orbits, spe, tb = I.space("pf")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    _, p = pivot(c.dim, 8, N.BS_F32)
    ev_full, rep_full = c.lanczos(p, 8, N.BS_F32, 80, 5, refine=True)
    ev, rep = c.lanczos(p, 8, N.BS_F32, 16, 5, refine=True, nthick=24, max_restarts=80, tol=1e-3)
    assert rep["restarts"] >= 1
    assert max(rep["residual"][:3]) <= 1e-3, rep
    assert np.max(np.abs(ev[:3] - ev_full[:3])) <= 1e-4, (ev, ev_full)
    ev_b, _ = c.lanczos(p, 8, N.BS_F32, 16, 5, refine=True, nthick=24, max_restarts=80, tol=1e-3)
    assert np.array_equal(ev, ev_b)
    c.sync_status()


@pytest.mark.gpu
def test_thick_restart_argument_checks(sd44):
    c, o = sd44
    _, pd = pivot(o.dim, 4, N.BS_F64)
    for kw in [dict(niter=8, nthick=6),                  # not a multiple of k
               dict(niter=8, nthick=28),                 # nthick / k + 1 >= niter
               dict(niter=8, nthick=-4),
               dict(niter=8, nthick=8, max_restarts=-1),
               dict(niter=8, nthick=8, tol=-1.0)]:
        niter = kw.pop("niter")
        with pytest.raises(N.BSError) as e:
            c.lanczos(pd, 4, N.BS_F64, niter, 3, refine=False, **kw)
        assert e.value.code == -1, kw


@pytest.mark.gpu
@pytest.mark.parametrize("idx,niter,restarts", [(8, 40, 60), (100, 60, 100)])
def test_targeted_thick_restart_finds_levels_nearest_target(idx, niter, restarts):
    """sd 2p2n (dim 640), FP64 k = 2: thick restart on (H - E_bar)^2 returns the
    three levels of H nearest E_bar (dense diagonalization of the oracle's
    H), as FP64 Rayleigh quotients with small residuals, like the oracle's
    targeted run; the graph-captured iteration gives the same levels."""
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 2, 2, 0, +1, device=0)
    o = O.Oracle(orbits, 2, 2, 0, 0).set_interaction(spe, tb)
    ev = np.linalg.eigvalsh(o.dense())
    Eb = 0.5 * (ev[idx] + ev[idx + 1]) + 0.013
    near = np.sort(ev[np.argsort(np.abs(ev - Eb))[:3]])
    ph, pd = pivot(o.dim, 2, N.BS_F64)
    e, rep = c.lanczos(pd, 2, N.BS_F64, niter, 3, refine=True, nthick=8, max_restarts=restarts, target=Eb)
    assert np.max(np.abs(np.sort(e) - near)) < 1e-8, (e, near)
    assert max(rep["residual"]) < 1e-6
    assert rep["matvec_blocks"] == 2 * (niter + rep["restarts"] * (niter - 4))
    e_o, _, X_o = o.block_lanczos_thick(ph, niter, 8, restarts, nkeep=3, return_vectors=True, target=Eb)
    H = o.matrix()
    rq = np.sort([X_o[:, m] @ (H @ X_o[:, m]) / (X_o[:, m] @ X_o[:, m]) for m in range(3)])
    assert np.max(np.abs(np.sort(e) - rq)) < 1e-8
    s = torch.cuda.Stream()
    e_g, _ = c.lanczos(pd, 2, N.BS_F64, niter, 3, refine=True, nthick=8, max_restarts=restarts, target=Eb,
                       use_graph=True, stream=s.cuda_stream)
    assert np.max(np.abs(np.sort(e_g) - np.sort(e))) < 1e-9
    c.sync_status()


@pytest.mark.gpu
def test_targeted_argument_checks(sd44):
    c, o = sd44
    _, pd = pivot(o.dim, 4, N.BS_F64)
    for kw in [dict(refine=False), dict(nkeep=9), dict(target=float("nan"))]:
        args = dict(refine=True, nkeep=3, target=-30.0)
        args.update(kw)
        nk = args.pop("nkeep")
        with pytest.raises(N.BSError) as e:
            c.lanczos(pd, 4, N.BS_F64, 8, nk, nthick=8, max_restarts=2, **args)
        assert e.value.code == -1, kw
