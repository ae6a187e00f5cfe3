"""GPU block Lanczos (bs_lanczos) against the FP64 oracle.

  * FP64, k = 1, sd 2p2n: lowest eigenvalues equal dense diagonalization of the
    oracle's explicit H (1e-9 MeV) and the Ritz vectors are eigenvectors.
  * FP64, k = 1, sd 4p4n (dim 28,503): equal to the oracle's own Lanczos from
    the same pivot, iteration by iteration the same Krylov space (1e-8 MeV).
  * rotational invariance on the GPU path: the M=1 spectrum sits inside M=0
    (FP64, every level checked).
  * (FP32-mixed levels against the oracle: test_gpu_fp32_vs_oracle.py.)
  * the host eigensolver of T against numpy.
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I

torch = pytest.importorskip("torch")


def ctx_oracle(name, Z, Nn, twoM, with_oracle=True):
    orbits, spe, tb = I.space(name)
    c = N.make(orbits, spe, tb, Z, Nn, twoM, +1, device=0)
    o = O.Oracle(orbits, Z, Nn, twoM, 0).set_interaction(spe, tb) if with_oracle else None
    return c, o


def pivot(dim, k, dtype):
    p = I.random_block(dim, k, seed=I.PIVOT_SEED)
    return torch.from_numpy(p).to("cuda", torch.float64 if dtype == N.BS_F64 else torch.float32)


def test_host_eigensolver_matches_numpy():
    rng = np.random.default_rng(3)
    for n in (1, 3, 17, 120):
        A = rng.standard_normal((n, n))
        A = A + A.T
        w, Z = N.debug_eigh(A, min(n, 6))
        assert np.max(np.abs(w - np.linalg.eigvalsh(A))) < 1e-12 * max(1, np.abs(w).max())
        assert np.max(np.abs(A @ Z - Z * w[:Z.shape[1]])) < 1e-11 * max(1, np.abs(w).max())


def test_banded_host_eigensolver_matches_numpy():
    rng = np.random.default_rng(4)
    for k, nb in ((1, 200), (2, 30), (4, 25), (8, 40)):
        n = k * nb
        T = np.zeros((n, n))
        for b in range(nb):
            A = rng.standard_normal((k, k))
            T[b * k:(b + 1) * k, b * k:(b + 1) * k] = A + A.T
            if b + 1 < nb:
                B = rng.standard_normal((k, k))   # full, as Lambda^1/2 Q^T of a Gram eig
                T[(b + 1) * k:(b + 2) * k, b * k:(b + 1) * k] = B
                T[b * k:(b + 1) * k, (b + 1) * k:(b + 2) * k] = B.T
        w, Z = N.debug_eigh_banded(T, 2 * k - 1 if k > 1 else 1, 10, 6)
        ref = np.linalg.eigvalsh(T)[:10]
        assert np.max(np.abs(w - ref)) < 1e-12 * np.max(np.abs(ref))
        assert np.max(np.abs(T @ Z - Z * w[:6])) < 1e-11 * np.max(np.abs(ref))
        assert np.max(np.abs(Z.T @ Z - np.eye(6))) < 1e-10


@pytest.mark.gpu
def test_fp64_lanczos_sd22_equals_dense():
    c, o = ctx_oracle("sd", 2, 2, 0)
    ev_d = np.linalg.eigvalsh(o.dense())[:5]
    evecs = torch.zeros((o.dim, 5), device="cuda", dtype=torch.float64)
    ev, rep = c.lanczos(pivot(o.dim, 1, N.BS_F64), 1, N.BS_F64, 200, 5, refine=True, evecs=evecs)
    assert np.max(np.abs(ev - ev_d)) < 1e-9, (ev, ev_d)
    X = evecs.cpu().numpy()
    H = o.matrix()
    for m in range(5):
        r = H @ X[:, m] - ev[m] * X[:, m]
        assert np.linalg.norm(r) < 1e-7
        assert rep["residual"][m] < 1e-7


@pytest.mark.gpu
def test_fp64_lanczos_sd44_equals_oracle_lanczos():
    c, o = ctx_oracle("sd", 4, 4, 0)
    p = pivot(o.dim, 1, N.BS_F64)
    ev, rep = c.lanczos(p, 1, N.BS_F64, 150, 10, refine=False)
    ev_o = o.lanczos(p.cpu().numpy()[:, 0], 150, nkeep=10)
    assert rep["iterations"] == 150
    assert np.max(np.abs(ev - ev_o)) < 1e-8, (ev, ev_o)


@pytest.mark.gpu
def test_fp32_block_lanczos_48cr_reproducible_and_within_1e4_mev():
    """48Cr (pf 4p4n, dim 1,963,461), FP32 k = 8, 80 block iterations: two runs
    give bit-identical eigenvalues (the streamed block products keep a fixed
    order and no stage of their rings is overwritten while read), the lowest
    three levels converge (FP64 residual <= 1e-3 MeV) and agree with FP64
    k = 1 Lanczos within 1e-4 MeV."""
    c, _ = ctx_oracle("pf", 4, 4, 0, with_oracle=False)
    p = pivot(c.dim, 8, N.BS_F32)
    ev_a, rep_a = c.lanczos(p, 8, N.BS_F32, 80, 5, refine=True)
    ev_b, _ = c.lanczos(p, 8, N.BS_F32, 80, 5, refine=True)
    assert np.array_equal(ev_a, ev_b)
    assert max(rep_a["residual"][:3]) <= 1e-3, rep_a["residual"]
    ev64, rep64 = c.lanczos(pivot(c.dim, 1, N.BS_F64), 1, N.BS_F64, 300, 5, refine=True)
    assert max(rep64["residual"][:3]) <= 1e-6
    assert np.max(np.abs(ev_a[:3] - ev64[:3])) <= 1e-4, (ev_a, ev64)
    c.sync_status()


@pytest.mark.gpu
def test_gpu_j_degeneracy_m1_inside_m0():
    c0, _ = ctx_oracle("sd", 4, 4, 0, with_oracle=False)
    c1, _ = ctx_oracle("sd", 4, 4, 2, with_oracle=False)
    e0, r0 = c0.lanczos(pivot(c0.dim, 1, N.BS_F64), 1, N.BS_F64, 300, 16, refine=True)
    e1, r1 = c1.lanczos(pivot(c1.dim, 1, N.BS_F64), 1, N.BS_F64, 300, 8, refine=True)
    # residuals <= 1e-4 MeV bound each level's error by r^2 / gap << 1e-6 MeV
    assert max(r0["residual"]) < 1e-4 and max(r1["residual"]) < 1e-4
    # each M=1 level is a distinct M=0 level (J >= 1 states appear in both); the
    # 16 lowest M=0 levels reach above the 8 lowest M=1 ones, so none escapes
    assert e1.max() < e0.max()
    left = list(e0)
    for e in np.sort(e1):
        j = int(np.argmin(np.abs(np.array(left) - e)))
        assert abs(left[j] - e) < 1e-6, (e, left)
        left.pop(j)


@pytest.mark.gpu
def test_breakdown_restart_and_exhaustion():
    # 1 proton + 1 neutron in the p shell, M=0: dim 10; ask for more
    # iterations than the space holds
    orbits, spe, tb = I.space("p")
    c = N.make(orbits, spe, tb, 1, 1, 0, +1, device=0)
    o = O.Oracle(orbits, 1, 1, 0, 0).set_interaction(spe, tb)
    ev, rep = c.lanczos(pivot(c.dim, 1, N.BS_F64), 1, N.BS_F64, 50, 3, refine=True)
    assert rep["iterations"] <= c.dim
    assert np.max(np.abs(ev - np.linalg.eigvalsh(o.dense())[:3])) < 1e-9


@pytest.mark.gpu
@pytest.mark.parametrize("k,dtype", [(1, N.BS_F64), (4, N.BS_F32), (8, N.BS_F32), (2, N.BS_F64)])
def test_block_dots_match_fp64_numpy(k, dtype):
    c, _ = ctx_oracle("sd", 4, 4, 0, with_oracle=False)
    nb = 5
    rng = np.random.default_rng(k)
    tdt = torch.float64 if dtype == N.BS_F64 else torch.float32
    V = torch.from_numpy(rng.standard_normal((nb, c.dim, k))).to("cuda", tdt)
    W = torch.from_numpy(rng.standard_normal((c.dim, k))).to("cuda", tdt)
    C = torch.zeros(nb * k * k, device="cuda", dtype=torch.float64)
    c.block_dots(V, nb, W, k, dtype, C)
    ref = np.einsum("bai,aj->bij", V.double().cpu().numpy(), W.double().cpu().numpy()).reshape(-1)
    got = C.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    C2 = torch.zeros_like(C)
    c.block_dots(V, nb, W, k, dtype, C2)
    assert torch.equal(C, C2)


@pytest.mark.gpu
@pytest.mark.parametrize("k,dtype", [(8, N.BS_F32), (4, N.BS_F32), (2, N.BS_F32), (1, N.BS_F32),
                                     (1, N.BS_F64), (2, N.BS_F64), (8, N.BS_F64)])
def test_block_dots_streamed_sizes(k, dtype):
    """Block inner products on sd 6p6n (dim 93,710): for k >= 2, or FP64, a
    block is a multiple of 16 bytes and the TMA-streamed kernel runs, with
    chunks of 2,048 elements spread over the CTAs (some get two, some none)
    and a ragged last chunk; FP32 k = 1 (374,840 bytes per block) takes the
    row-slot kernel.  Against FP64 numpy, and bit-identical when repeated."""
    c, _ = ctx_oracle("sd", 6, 6, 0, with_oracle=False)
    assert c.dim == 93710
    nb = 7
    rng = np.random.default_rng(40 + k)
    tdt = torch.float64 if dtype == N.BS_F64 else torch.float32
    V = torch.from_numpy(rng.standard_normal((nb, c.dim, k))).to("cuda", tdt)
    W = torch.from_numpy(rng.standard_normal((c.dim, k))).to("cuda", tdt)
    C = torch.zeros(nb * k * k, device="cuda", dtype=torch.float64)
    c.block_dots(V, nb, W, k, dtype, C)
    ref = np.einsum("bai,aj->bij", V.double().cpu().numpy(), W.double().cpu().numpy()).reshape(-1)
    got = C.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    C2 = torch.zeros_like(C)
    c.block_dots(V, nb, W, k, dtype, C2)
    assert torch.equal(C, C2)
    c.sync_status()   # raises on a recorded wait timeout


@pytest.mark.gpu
@pytest.mark.parametrize("space,Z,k,dtype,nb", [("sd", 6, 8, N.BS_F32, 7), ("sd", 6, 4, N.BS_F32, 5),
                                              ("sd", 6, 2, N.BS_F32, 3), ("sd", 6, 1, N.BS_F32, 9),
                                              ("sd", 6, 1, N.BS_F64, 4), ("sd", 6, 8, N.BS_F64, 2),
                                              ("pf", 4, 8, N.BS_F32, 3), ("pf", 4, 1, N.BS_F64, 2)])
def test_block_update_matches_fp64_numpy(space, Z, k, dtype, nb):
    """W -= sum_b V_b C_b against FP64 numpy: sd 6p6n and pf 4p4n (48Cr, ragged
    last tile of the streamed kernel), every k, FP32 and FP64, and the
    row-slot kernel where a block is not a multiple of 16 bytes (FP32 k = 1
    at dim 93,710 and 1,963,461)."""
    c, _ = ctx_oracle(space, Z, Z, 0, with_oracle=False)
    rng = np.random.default_rng(70 + k + nb)
    tdt = torch.float64 if dtype == N.BS_F64 else torch.float32
    V = torch.from_numpy(rng.standard_normal((nb, c.dim, k))).to("cuda", tdt)
    W = torch.from_numpy(rng.standard_normal((c.dim, k))).to("cuda", tdt)
    Cm = rng.standard_normal((nb, k, k)) * 0.1
    C = torch.from_numpy(Cm.reshape(-1)).to("cuda", torch.float64)
    Vh, Wh = V.double().cpu().numpy(), W.double().cpu().numpy()
    Ch = Cm.astype(np.float32).astype(np.float64) if dtype == N.BS_F32 else Cm   # used in the vectors' precision
    ref = Wh - np.einsum("bai,bij->aj", Vh, Ch)
    bound = np.abs(Wh) + np.einsum("bai,bij->aj", np.abs(Vh), np.abs(Ch))
    c.block_update(V, nb, C, W, k, dtype)
    torch.cuda.synchronize()
    got = W.double().cpu().numpy()
    tol = 1e-13 if dtype == N.BS_F64 else (nb * k + 1) * 2.0 ** -23
    assert np.all(np.abs(got - ref) <= tol * bound)
    c.sync_status()


@pytest.mark.gpu
@pytest.mark.parametrize("k,dtype", [(1, N.BS_F64), (8, N.BS_F32)])
def test_graph_captured_iteration_equals_plain_loop(k, dtype):
    c, _ = ctx_oracle("sd", 4, 4, 0, with_oracle=False)
    s = torch.cuda.Stream()
    p = pivot(c.dim, k, dtype)
    torch.cuda.synchronize()
    ev_a, rep_a = c.lanczos(p, k, dtype, 40, 4, refine=True, stream=s.cuda_stream)
    ev_b, rep_b = c.lanczos(p, k, dtype, 40, 4, refine=True, stream=s.cuda_stream, use_graph=True)
    assert rep_b["iterations"] == rep_a["iterations"] == 40
    assert np.max(np.abs(ev_a - ev_b)) <= 1e-12 * np.max(np.abs(ev_a))
    ev_c, rep_c = c.lanczos(p, k, dtype, 40, 4, refine=True, use_graph=True)   # default stream -> own stream
    assert np.max(np.abs(ev_a - ev_c)) <= 1e-12 * np.max(np.abs(ev_a))
