"""bs_block_dots_noalloc: the block inner products for callers that cannot
allocate device memory (its partial sums live in a fixed device array the
library carries), checked against bs_block_dots, the entry point that
allocates its partials, on two calls in a row with different inputs.

This file is collected last so that a run stopping at the first failure has
run every other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_08432_gb300 import _native as N  # noqa: E402
from paper_1801_08432_gb300 import build as B  # noqa: E402
from paper_1801_08432_gb300 import inputs as I  # noqa: E402


@pytest.mark.parametrize("k,dtype", [(1, N.BS_F64), (8, N.BS_F32), (4, N.BS_F32), (2, N.BS_F64)])
def test_noalloc_block_dots_match_allocating_entry_point(k, dtype):
    B.build()
    L = N.load()
    orbits, spe, tb = I.space("sd")
    c = N.make(orbits, spe, tb, 4, 4, 0, +1, device=0)
    dim, nb = c.dim, 6
    tdt = torch.float64 if dtype == N.BS_F64 else torch.float32
    stream = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(100 + k)
    for call in range(2):   # two calls in a row, different inputs
        V = torch.from_numpy(rng.standard_normal((nb, dim, k))).to("cuda", tdt)
        W = torch.from_numpy(rng.standard_normal((dim, k))).to("cuda", tdt)
        ref = torch.zeros(nb * k * k, device="cuda", dtype=torch.float64)
        c.block_dots(V, nb, W, k, dtype, ref, stream)
        out = torch.full((nb * k * k,), float("nan"), device="cuda", dtype=torch.float64)
        rc = L.bs_block_dots_noalloc(ctypes.c_void_p(V.data_ptr()), nb, ctypes.c_void_p(W.data_ptr()), dim, k, dtype,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0, call
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o)), call
        assert np.max(np.abs(o - r)) <= 1e-12 * np.max(np.abs(r)), call


@pytest.mark.parametrize("k,dtype,nb", [(8, N.BS_F32, 14), (8, N.BS_F32, 4096), (2, N.BS_F64, 4096)])
def test_noalloc_block_dots_on_fewer_ctas(k, dtype, nb):
    """Requests too large for two partial blocks per SM run on fewer CTAs:
    nb * k * k just above the fixed capacity / (2 x SMs), and exactly at the
    capacity (nb = 4096 at k = 8: one CTA fills the whole array).  Checked
    against FP64 products, twice in a row."""
    B.build()
    L = N.load()
    dim = 640
    tdt = torch.float64 if dtype == N.BS_F64 else torch.float32
    stream = torch.cuda.current_stream().cuda_stream
    g = torch.Generator(device="cuda").manual_seed(7 + nb)
    for call in range(2):
        V = torch.randn((nb, dim, k), device="cuda", dtype=tdt, generator=g)
        W = torch.randn((dim, k), device="cuda", dtype=tdt, generator=g)
        ref = torch.einsum("bai,aj->bij", V.double(), W.double()).reshape(-1)
        out = torch.full((nb * k * k,), float("nan"), device="cuda", dtype=torch.float64)
        rc = L.bs_block_dots_noalloc(ctypes.c_void_p(V.data_ptr()), nb, ctypes.c_void_p(W.data_ptr()), dim, k, dtype,
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
        assert rc == 0, call
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o)), call
        assert np.max(np.abs(o - r)) <= 1e-12 * np.max(np.abs(r)), call


def test_noalloc_rejects_oversize_and_bad_arguments():
    B.build()
    L = N.load()
    x = torch.zeros((16, 8), device="cuda", dtype=torch.float32)
    C = torch.zeros(64, device="cuda", dtype=torch.float64)
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    too_many = 262144 // 64 + 1                         # nb * 8 * 8 above the fixed capacity
    assert L.bs_block_dots_noalloc(p(x), too_many, p(x), 16, 8, N.BS_F32, p(C), None) == -4   # BS_ENOMEM
    assert L.bs_block_dots_noalloc(p(x), 1, p(x), 16, 3, N.BS_F32, p(C), None) == -1          # k = 3
    assert L.bs_block_dots_noalloc(None, 1, p(x), 16, 8, N.BS_F32, p(C), None) == -1
    # pointers the kernel's 16-byte loads would fault on are refused on the host
    # (nothing is launched): FP32 k = 8 at a 4-byte offset, FP64 k = 2 at 8
    off = lambda t, b: ctypes.c_void_p(t.data_ptr() + b)
    assert L.bs_block_dots_noalloc(off(x, 4), 1, p(x), 15, 8, N.BS_F32, p(C), None) == -1
    assert L.bs_block_dots_noalloc(p(x), 1, off(x, 4), 15, 8, N.BS_F32, p(C), None) == -1
    assert L.bs_block_dots_noalloc(p(x), 1, p(x), 15, 8, N.BS_F32, off(C, 4), None) == -1
    assert L.bs_block_dots_noalloc(off(x, 8), 1, p(x), 7, 2, N.BS_F64, p(C), None) == -1
    # FP32 k = 1 needs only 4-byte alignment: an odd element offset is accepted
    assert L.bs_block_dots_noalloc(off(x, 4), 1, p(x), 15, 1, N.BS_F32, p(C), None) == 0
    torch.cuda.synchronize()
