"""GPU parity of y = H x (the fused CUDA kernel, through the C ABI) against the
FP64 oracle.

Full vectors on spaces the oracle's explicit matrix covers in seconds (sd
2p2n, 4p4n, 6p6n at M=0 and M=1, edge cases), and sampled rows computed on
the fly by the oracle at the full sizes (pf 4p4n, dim 1,963,461; pf 6p6n,
dim 109,954,620) in the launch configuration the benchmark times.

Tolerances.  FP64: max|dy| <= 1e-12 * max|y| (the stated FP64 bar).  FP32
(vectors, coefficients and accumulation in float): each output is a sum of n
products; the rounding error is bounded by about n * 2^-24 * (|H| |x|)_i, n up
to ~10^3 here, so the test uses max|dy_i| <= 4e-5 * max_i (|H| |x|)_i and
reports the typical error.
"""
import numpy as np
import pytest

import oracle as O
from paper_1801_08432_gb300 import _native as N
from paper_1801_08432_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_cache = {}


def setup(name, Z, Nn, twoM, parity=+1):
    key = (name, Z, Nn, twoM, parity)
    if key not in _cache:
        orbits, spe, tb = I.space(name)
        c = N.make(orbits, spe, tb, Z, Nn, twoM, parity, device=0)
        o = O.Oracle(orbits, Z, Nn, twoM, 0 if parity > 0 else 1).set_interaction(spe, tb)
        _cache[key] = (c, o)
    return _cache[key]


def gpu_apply(c, x, k, dtype):
    tdt = torch.float64 if dtype == N.BS_F64 else torch.float32
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=tdt)
    yd = torch.full_like(xd, float("nan"))
    c.apply_H(xd, yd, k, dtype, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return yd.double().cpu().numpy()


SMALL = [("sd", 2, 2, 0), ("sd", 4, 4, 0), ("sd", 4, 4, 2), ("sd", 6, 6, 0), ("sd", 6, 6, 2),
         ("sd", 1, 1, 0), ("sd", 2, 0, 0), ("sd", 0, 3, 3), ("sd", 5, 6, 1), ("p", 4, 4, 0), ("pf", 2, 2, 0)]


@pytest.mark.parametrize("case", SMALL, ids=lambda c: "%s-%dp%dn-2M%d" % c)
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_fp64_full_vector(case, k):
    c, o = setup(*case)
    x = I.random_block(o.dim, k, seed=k)
    y = gpu_apply(c, x, k, N.BS_F64)
    ref = o.spmv(x)
    assert np.all(np.isfinite(y))
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("case", [("sd", 4, 4, 0), ("sd", 6, 6, 0), ("sd", 5, 6, 1)], ids=lambda c: "%s-%dp%dn-2M%d" % c)
@pytest.mark.parametrize("k", [1, 4, 8])
def test_fp32_full_vector(case, k):
    c, o = setup(*case)
    x = I.random_block(o.dim, k, seed=10 + k)
    y = gpu_apply(c, x.astype(np.float32), k, N.BS_F32)
    ref = o.spmv(x.astype(np.float32).astype(np.float64))
    H = o.matrix()
    absref = abs(H) @ np.abs(x.astype(np.float32).astype(np.float64))
    assert np.all(np.abs(y - ref) <= 4e-5 * absref + 1e-30)


def test_deterministic_and_k_consistent():
    c, o = setup("sd", 6, 6, 0)
    x = I.random_block(o.dim, 4, seed=3)
    y1 = gpu_apply(c, x, 4, N.BS_F64)
    y2 = gpu_apply(c, x, 4, N.BS_F64)
    assert np.array_equal(y1, y2)
    # the k columns are independent products; the staging chunk size (and so
    # the summation order) depends on k, so equality is to rounding
    for col in range(4):
        yc = gpu_apply(c, x[:, col:col + 1].copy(), 1, N.BS_F64)
        assert np.max(np.abs(yc[:, 0] - y1[:, col])) <= 1e-14 * np.max(np.abs(y1))


def test_host_buffer_entry_point():
    c, o = setup("sd", 4, 4, 0)
    x = I.random_block(o.dim, 2, seed=5)
    y = np.zeros_like(x)
    c.apply_H_host(x, y, 2, N.BS_F64)
    assert np.array_equal(y, gpu_apply(c, x, 2, N.BS_F64))


def test_host_buffer_entry_point_pinned_and_pageable():
    """sd 6p6n, k = 8 FP32 (3.0 MB per vector block), page-locked and pageable
    host buffers, twice in a row: the same y as the device-buffer call."""
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 6, 6, 0, +1, device=0)
    x = I.random_block(c.dim, 8, seed=7).astype(np.float32)
    ref = gpu_apply(c, x, 8, N.BS_F32)
    xp = torch.from_numpy(x).pin_memory()
    yp = torch.zeros_like(xp).pin_memory()
    for _ in range(2):
        y = np.full_like(x, np.nan)
        c.apply_H_host(x, y, 8, N.BS_F32)            # pageable
        assert np.array_equal(y, ref)
        yp.fill_(float("nan"))
        c.apply_H_host(xp.numpy(), yp.numpy(), 8, N.BS_F32)   # page-locked
        assert np.array_equal(yp.numpy(), ref)
    c.close()


def test_async_host_entry_point_two_streams_two_slots():
    """bs_apply_H_host_async: six calls alternating two streams and the two
    staging slots, each with its own input block (pinned), synchronized only at
    the end: every result equals the device-buffer product bit for bit (FP32
    k = 8 and 4, FP64 k = 1 on sd 6p6n); slots other than 0 and 1 are
    rejected before anything is enqueued."""
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 6, 6, 0, +1, device=0)
    sts = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k, dt, npt in ((8, N.BS_F32, np.float32), (4, N.BS_F32, np.float32), (1, N.BS_F64, np.float64)):
        xs = [torch.from_numpy(I.random_block(c.dim, k, seed=20 + i).astype(npt)).pin_memory() for i in range(6)]
        ys = [torch.full_like(x, float("nan")).pin_memory() for x in xs]
        for i in range(6):
            c.apply_H_host_async(xs[i], ys[i], k, dt, sts[i % 2].cuda_stream, i % 2)
        for st in sts:
            st.synchronize()
        for i in range(6):
            assert np.array_equal(ys[i].numpy(), gpu_apply(c, xs[i].numpy(), k, dt)), (k, i)
    x = torch.zeros((c.dim, 1), dtype=torch.float64).pin_memory()
    for slot in (-1, 2):
        with pytest.raises(N.BSError):
            c.apply_H_host_async(x, x.clone(), 1, N.BS_F64, 0, slot)
    c.close()


def test_rejects_bad_calls():
    c, o = setup("sd", 2, 2, 0)
    xd = torch.zeros((o.dim, 3), device="cuda", dtype=torch.float64)
    yd = torch.zeros_like(xd)
    with pytest.raises(N.BSError):
        c.apply_H(xd, yd, 3, N.BS_F64)       # k = 3
    with pytest.raises(N.BSError):
        c.apply_H(xd, xd, 1, N.BS_F64)       # aliasing
    with pytest.raises(N.BSError):
        c.apply_H(xd, yd, 1, 7)              # dtype


def _sample_rows(o, n, seed):
    rng = np.random.default_rng(seed)
    B = o.basis()
    edges = []
    for (_, _, off) in B["blocks"]:
        edges += [off, max(off - 1, 0)]
    edges.append(o.dim - 1)
    rows = np.unique(np.concatenate([rng.integers(0, o.dim, n), np.array(edges, dtype=np.int64)]))
    return rows


@pytest.mark.parametrize("k,dtype", [(1, N.BS_F64), (8, N.BS_F64), (8, N.BS_F32), (4, N.BS_F32)])
def test_pf_4p4n_sampled_rows(k, dtype):
    c, o = setup("pf", 4, 4, 0)
    assert o.dim == 1963461
    x = I.random_block(o.dim, k, seed=21)
    if dtype == N.BS_F32:
        x = x.astype(np.float32).astype(np.float64)
    y = gpu_apply(c, x, k, dtype)
    rows = _sample_rows(o, 6000, 1)
    ref = o.apply_rows(rows, x)
    err = np.max(np.abs(y[rows] - ref))
    if dtype == N.BS_F64:
        assert err <= 1e-12 * np.max(np.abs(y))
    else:
        bound = o.apply_rows(rows, np.abs(x), absval=True)
        assert np.all(np.abs(y[rows] - ref) <= 4e-5 * bound + 1e-30)
    assert np.all(np.isfinite(y))


@pytest.mark.parametrize("mode", [17, 18, 19, 20])
def test_pf_6p6n_core_grouped_modes(mode):
    """The core-grouped pn path at the pf 6p6n size (neutron sectors up to
    3,952 columns, source rows of 63 KB at k = 4), with the like-particle terms
    on the first pipelined variant that fits (17, 18) or the nn term in
    2-row tiles of 576-column tiles (19): sampled rows against the oracle and
    a bit-identical repeat."""
    c, o = setup("pf", 6, 6, 0)
    k = 4
    g = torch.Generator(device="cuda").manual_seed(11)
    xd = torch.randn((o.dim, k), device="cuda", dtype=torch.float32, generator=g)
    yd, yd2 = torch.empty_like(xd), torch.empty_like(xd)
    s = torch.cuda.current_stream().cuda_stream
    c.set_kernel(mode)
    try:
        c.apply_H(xd, yd, k, N.BS_F32, s)
        c.apply_H(xd, yd2, k, N.BS_F32, s)
        torch.cuda.synchronize()
        c.sync_status()
    finally:
        c.set_kernel(0)
    assert torch.equal(yd, yd2)
    rows = _sample_rows(o, 1500, 4)
    x = xd.double().cpu().numpy()
    ref = o.apply_rows(rows, x)
    bound = o.apply_rows(rows, np.abs(x), absval=True)
    y = yd[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert np.all(np.abs(y - ref) <= 4e-5 * bound + 1e-30)


@pytest.mark.parametrize("k,dtype", [(4, N.BS_F32), (1, N.BS_F64)])
def test_pf_6p6n_sampled_rows(k, dtype):
    c, o = setup("pf", 6, 6, 0)
    assert o.dim == 109954620
    dt = torch.float64 if dtype == N.BS_F64 else torch.float32
    g = torch.Generator(device="cuda").manual_seed(7)
    xd = torch.randn((o.dim, k), device="cuda", dtype=dt, generator=g)
    yd = torch.empty_like(xd)
    c.apply_H(xd, yd, k, dtype, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    rows = _sample_rows(o, 1500, 2)
    x = xd.double().cpu().numpy()
    ref = o.apply_rows(rows, x)
    y = yd[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    scale = np.max(np.abs(ref))
    if dtype == N.BS_F64:
        assert np.max(np.abs(y - ref)) <= 1e-12 * scale
    else:
        bound = o.apply_rows(rows, np.abs(x), absval=True)
        assert np.all(np.abs(y - ref) <= 4e-5 * bound + 1e-30)


@pytest.mark.parametrize("case", [("sd", 4, 4, 0), ("sd", 5, 6, 1), ("sd", 0, 3, 3), ("pf", 2, 2, 0)],
                         ids=lambda c: "%s-%dp%dn-2M%d" % c)
@pytest.mark.parametrize("k", [1, 2, 4, 8])
def test_row_and_tiled_kernels_agree_with_oracle(case, k):
    c, o = setup(*case)
    x = I.random_block(o.dim, k, seed=30 + k)
    ref = o.spmv(x)
    for mode in list(range(1, N.KERNEL_MODES + 1)) + [0]:
        c.set_kernel(mode)
        y = gpu_apply(c, x, k, N.BS_F64)
        c.sync_status()
        assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref)), mode
    c.set_kernel(0)
    xf = x.astype(np.float32)
    for mode in range(1, N.KERNEL_MODES + 1):
        c.set_kernel(mode)
        yf = gpu_apply(c, xf, k, N.BS_F32)
        c.sync_status()
        bound = abs(o.matrix()) @ np.abs(xf.astype(np.float64))
        assert np.all(np.abs(yf - ref) <= 4e-5 * bound + 1e-6 * np.max(np.abs(ref)))
    c.set_kernel(0)


def test_autotune_picks_a_valid_mode():
    c, o = setup("sd", 6, 6, 0)
    s = torch.cuda.current_stream().cuda_stream
    for k, dt in ((1, N.BS_F64), (8, N.BS_F32)):
        m = c.autotune(k, dt, s)
        assert 1 <= m <= N.KERNEL_MODES
    x = I.random_block(o.dim, 8, seed=4).astype(np.float32)
    y = gpu_apply(c, x, 8, N.BS_F32)
    ref = o.spmv(x.astype(np.float64))
    assert np.max(np.abs(y - ref)) <= 1e-5 * np.max(np.abs(ref)) * 10
    c.sync_status()


@pytest.mark.parametrize("mode", [11, 12, 13, 14, 15, 16, 17, 18, 19, 20])
@pytest.mark.parametrize("k", [4, 8])
def test_pf_4p4n_core_grouped_modes(mode, k):
    """The core-grouped pn path (FP32, k = 4, 8) at the benchmark size: sampled
    rows against the oracle, bit-identical repeats, and agreement with the
    pipelined kernel to FP32 rounding."""
    c, o = setup("pf", 4, 4, 0)
    x = I.random_block(o.dim, k, seed=23).astype(np.float32)
    c.set_kernel(mode)
    try:
        y = gpu_apply(c, x, k, N.BS_F32)
        y2 = gpu_apply(c, x, k, N.BS_F32)
        c.sync_status()
        c.set_kernel(6)
        yp = gpu_apply(c, x, k, N.BS_F32)
    finally:
        c.set_kernel(0)
    assert np.array_equal(y, y2)
    rows = _sample_rows(o, 4000, 3)
    x64 = x.astype(np.float64)
    ref = o.apply_rows(rows, x64)
    bound = o.apply_rows(rows, np.abs(x64), absval=True)
    assert np.all(np.abs(y[rows] - ref) <= 4e-5 * bound + 1e-30)
    assert np.max(np.abs(y - yp)) <= 1e-5 * np.max(np.abs(yp))


@pytest.mark.gpu
def test_set_tuned_replays_a_mode_and_rejects_bad_arguments():
    """bs_set_tuned records a mode for (k, dtype) without timing; mode-0 calls
    then run it (the product equals the one with the mode forced)."""
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    x = torch.from_numpy(I.random_block(c.dim, 8, seed=3)).to("cuda", torch.float32)
    y_set, y_forced = torch.empty_like(x), torch.empty_like(x)
    c.set_tuned(8, N.BS_F32, 13)
    c.apply_H(x, y_set, 8, N.BS_F32)
    c.set_kernel(13)
    c.apply_H(x, y_forced, 8, N.BS_F32)
    c.set_kernel(0)
    torch.cuda.synchronize()
    assert torch.equal(y_set, y_forced)
    for bad in ((3, N.BS_F32, 13), (8, 7, 13), (8, N.BS_F32, 0), (8, N.BS_F32, N.KERNEL_MODES + 1)):
        with pytest.raises(Exception):
            c.set_tuned(*bad)
    c.close()


@pytest.mark.gpu
def test_gather_ceiling_is_measured_and_ordered():
    """bs_gather_ceiling: positive rates, below the FP32 FMA-issue rate of the
    device, and more FLOP/s when each gathered element feeds more rows."""
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 2, 2, 0, +1, device=0)
    props = torch.cuda.get_device_properties(0)
    issue = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e9   # GFLOP/s at a 2.2 GHz upper clock
    for where in (0, 1):
        g = [c.gather_ceiling(where, 8, r) for r in (1, 2, 4)]
        assert all(0 < x < issue for x in g), g
        # each doubling of the rows fed per gather raises the rate by a factor in
        # [1.4, 2.1]: the gathers stay the same, the FMAs per gather double (a
        # microbenchmark that lost its gathers or its FMAs would fall outside)
        assert 1.4 <= g[1] / g[0] <= 2.1 and 1.4 <= g[2] / g[1] <= 2.1, g
    with pytest.raises(N.BSError):
        c.gather_ceiling(2, 8, 1)
    c.close()


def test_pn_core_kernel_stays_below_its_gather_ceiling():
    """The dominant kernel of the 48Cr k = 8 product (the pn term by proton
    cores, mode 20) against the measured shared-memory ceiling at its own
    rows per gathered element (multiply-adds / gathers, both counted in the
    tables), interpolated between the measured 2- and 4-row rates: a kernel
    faster than that ceiling would mean the ceiling does not bound it."""
    c, _ = setup("pf", 4, 4, 0)
    stats = c.table("stats", np.int64)
    fma, gathers = float(stats[8]), float(stats[11])
    rpg = fma / gathers
    assert 1.0 <= rpg <= 4.0
    g2, g4 = (c.gather_ceiling(0, 8, r) / 1e3 for r in (2, 4))
    lo, hi, clo, chi = (2, 4, g2, g4) if rpg >= 2 else (1, 2, c.gather_ceiling(0, 8, 1) / 1e3, g2)
    ceiling = clo + (rpg - lo) / (hi - lo) * (chi - clo)
    x = torch.randn((c.dim, 8), device="cuda", dtype=torch.float32, generator=torch.Generator(device="cuda").manual_seed(3))
    y = torch.empty_like(x)
    c.set_kernel(20)
    try:
        for _ in range(2):
            c.apply_H(x, y, 8, N.BS_F32)
        c.time_kernel(5)
        for _ in range(5):
            c.apply_H(x, y, 8, N.BS_F32)
        ms = float(np.mean(c.kernel_times()))
        c.time_kernel(0)
    finally:
        c.set_kernel(0)
    tflops = 2.0 * fma * 8 / (ms / 1e3) / 1e12
    print("pn-core kernel %.3f ms, %.2f TFLOP/s, ceiling at %.3f rows per gather %.2f TFLOP/s, fraction %.3f"
          % (ms, tflops, rpg, ceiling, tflops / ceiling))
    assert 0.1 * ceiling < tflops <= 1.05 * ceiling
