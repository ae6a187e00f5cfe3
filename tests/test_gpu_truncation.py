"""W-truncated spaces (Sec. "Truncation of the many-body space") on the GPU,
against the FP64 oracle's truncated Hamiltonian (its full H restricted to the
states with W_p + W_n <= W_min + max_excite; states matched by bitstrings,
since the library orders the truncated basis by (2M, parity, W) sectors):

  * H x for k = 1, 2, 4, 8: FP64 within 1e-12 of max|y|, FP32 within
    4e-5 (|H||x|)_i element by element; sd and pf particle-hole weights at 0
    to 4 excitations, odd A with negative parity, uneven weights; every
    kernel mode falls back to the tiled kernel, which reads the
    like-particle moves that change W from other blocks;
  * eigenvalues: FP64 Lanczos equal to dense diagonalization of the
    truncated H (1e-9 MeV), FP32-mixed block Lanczos within 1e-4 MeV, and the
    M = 1 levels inside the M = 0 ones at a truncation;
  * 48Cr (pf 4p4n) with 1p-1h and 2p-2h truncations: sampled rows of H x
    against the oracle's on-the-fly rows of the full H applied to x placed
    in the kept states (zero elsewhere).
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I
from tests.test_truncation import SPACES, _tbmes, lib_states, oracle_case

torch = pytest.importorskip("torch")

CASES = [("sd", 4, 4, 0, +1, 0), ("sd", 4, 4, 0, +1, 1), ("sd", 4, 4, 0, +1, 2), ("pf", 2, 2, 0, +1, 2),
         ("pf", 3, 2, 1, -1, 2), ("sd_uneven", 3, 3, 0, +1, 4)]


def gpu_case(name, Z, Nn, twoM, par, mx):
    orbits, spe = SPACES[name]
    return N.make(orbits, spe, _tbmes(name), Z, Nn, twoM, par, device=0, max_excite=mx)


def mapped(o, mask, c):
    """Library index -> position among the oracle's kept states."""
    P, Q = lib_states(c)
    Po, Qo = o.states()
    idx = np.nonzero(mask)[0]
    pos = {(int(a), int(b)): j for j, (a, b) in enumerate(zip(Po[idx], Qo[idx]))}
    return np.array([pos[(int(a), int(b))] for a, b in zip(P, Q)])


@pytest.mark.gpu
@pytest.mark.parametrize("case", CASES, ids=lambda c: "%s-%dp%dn-2M%d-par%+d-x%d" % c)
def test_truncated_hx_equals_oracle(case):
    name, Z, Nn, twoM, par, mx = case
    o, mask, _ = oracle_case(*case)
    orbits, _ = SPACES[name]
    H = o.truncated_matrix([x.w for x in orbits], mx)
    c = gpu_case(*case)
    perm = mapped(o, mask, c)
    for mode in (0, 2, 6, 13):
        c.set_kernel(mode)
        for k in (1, 2, 4, 8):
            x = I.random_block(c.dim, k, seed=11 + k)
            xo = np.zeros_like(x)
            xo[perm] = x
            ref = (H @ xo)[perm]
            bound = (abs(H) @ np.abs(xo))[perm]
            for dt, tdt in ((N.BS_F64, torch.float64), (N.BS_F32, torch.float32)):
                xd = torch.from_numpy(x).to("cuda", tdt)
                yd = torch.full_like(xd, float("nan"))
                c.apply_H(xd, yd, k, dt)
                torch.cuda.synchronize()
                y = yd.double().cpu().numpy()
                if dt == N.BS_F64:
                    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref)), (mode, k)
                else:
                    assert np.all(np.abs(y - ref) <= 4e-5 * bound + 1e-30), (mode, k)
    c.sync_status()


@pytest.mark.gpu
@pytest.mark.parametrize("case", [("sd", 4, 4, 0, +1, 2), ("pf", 2, 2, 0, +1, 2), ("pf", 3, 2, 1, -1, 2)],
                         ids=lambda c: "%s-%dp%dn-2M%d-par%+d-x%d" % c)
def test_truncated_levels_equal_dense(case):
    name, Z, Nn, twoM, par, mx = case
    o, mask, _ = oracle_case(*case)
    orbits, _ = SPACES[name]
    ev_d = np.linalg.eigvalsh(o.truncated_matrix([x.w for x in orbits], mx).toarray())[:6]
    c = gpu_case(*case)
    p64 = torch.from_numpy(I.random_block(c.dim, 1, seed=I.PIVOT_SEED)).to("cuda", torch.float64)
    ev, rep = c.lanczos(p64, 1, N.BS_F64, min(300, c.dim), 6, refine=True)
    assert np.max(np.abs(ev - ev_d)) <= 1e-9, (ev, ev_d)
    p32 = torch.from_numpy(I.random_block(c.dim, 4, seed=I.PIVOT_SEED)).to("cuda", torch.float32)
    ev32, rep32 = c.lanczos(p32, 4, N.BS_F32, min(100, c.dim // 4), 6, refine=True)
    assert np.max(np.abs(ev32 - ev_d)) <= 1e-4, (ev32, ev_d, rep32["residual"])
    c.sync_status()


@pytest.mark.gpu
def test_truncated_m1_levels_inside_m0():
    c0 = gpu_case("pf", 2, 2, 0, +1, 2)
    c1 = gpu_case("pf", 2, 2, 2, +1, 2)
    e = []
    for c, n in ((c0, 16), (c1, 8)):
        p = torch.from_numpy(I.random_block(c.dim, 1, seed=I.PIVOT_SEED)).to("cuda", torch.float64)
        ev, rep = c.lanczos(p, 1, N.BS_F64, min(400, c.dim), n, refine=True)
        assert max(rep["residual"]) < 1e-6
        e.append(ev)
    e0, e1 = e
    assert e1.max() < e0.max()
    left = list(e0)
    for v in np.sort(e1):
        j = int(np.argmin(np.abs(np.array(left) - v)))
        assert abs(left[j] - v) < 1e-6, (v, left)
        left.pop(j)


@pytest.mark.gpu
@pytest.mark.parametrize("mx", [1, 2, 4])
def test_truncated_48cr_sampled_rows(mx):
    orbits, spe = SPACES["pf"]
    tb = _tbmes("pf")
    o = O.Oracle(orbits, 4, 4, 0, 0).set_interaction(spe, tb)
    mask, _, _ = o.truncation_mask([x.w for x in orbits], mx)
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0, max_excite=mx)
    assert c.dim == int(mask.sum())
    perm = mapped(o, mask, c)
    full = np.nonzero(mask)[0][perm]          # library index -> index in the full basis
    k = 4
    x = I.random_block(c.dim, k, seed=48)
    xf = np.zeros((o.dim, k))
    xf[full] = x
    rng = np.random.default_rng(mx)
    B = c.export_basis()
    rows = set(rng.integers(0, c.dim, 1500).tolist())
    for (ps, ns_, off) in B["blocks"]:
        rows.update((int(off), int(off + B["p_sec"][ps][3] * B["n_sec"][ns_][3] - 1)))
    rows = np.array(sorted(rows))
    ref = o.apply_rows(full[rows], xf)
    bound = o.apply_rows(full[rows], xf, absval=True)
    for dt, tdt in ((N.BS_F64, torch.float64), (N.BS_F32, torch.float32)):
        xd = torch.from_numpy(x).to("cuda", tdt)
        yd = torch.full_like(xd, float("nan"))
        c.apply_H(xd, yd, k, dt)
        torch.cuda.synchronize()
        y = yd.double().cpu().numpy()[rows]
        if dt == N.BS_F64:
            assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))
        else:
            assert np.all(np.abs(y - ref) <= 4e-5 * bound + 1e-30)
    c.sync_status()


@pytest.mark.gpu
def test_truncated_basis_rejects_backward_and_density():
    c = gpu_case("sd", 4, 4, 0, +1, 1)
    x = torch.zeros((c.dim, 1), device="cuda", dtype=torch.float64)
    with pytest.raises(N.BSError) as e:
        c.apply_H_backward(x, x, torch.zeros_like(x), 1, N.BS_F64, n_theta=3 + 63)
    assert e.value.code == -1
    with pytest.raises(N.BSError) as e:
        c.density(x, x, 1, 12)
    assert e.value.code == -1
