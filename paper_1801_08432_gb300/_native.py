"""ctypes binding of libbsgpu.so (include/bigstick_gpu.h), same names as the C ABI.

Argument marshalling only: every step of H*x, its adjoint and the Lanczos
driver runs in the library's CUDA kernels.  The library must have been built
(``paper_1801_08432_gb300.build.build()``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbsgpu.so")

BS_F64, BS_F32 = 0, 1
KERNEL_MODES = 20          # BS_KERNEL_MODES: selectable H x kernel modes 1..20
ERRORS = {0: "BS_OK", -1: "BS_EINVAL", -2: "BS_ENOBASIS", -3: "BS_ENOINT", -4: "BS_ENOMEM",
          -5: "BS_ECUDA", -6: "BS_EBREAKDOWN", -7: "BS_ETIMEOUT"}

# every symbol include/bigstick_gpu.h declares
EXPORTED = ["bs_create", "bs_destroy", "bs_last_error", "bs_build_basis", "bs_basis_info",
            "bs_export_basis", "bs_load_interaction", "bs_apply_H", "bs_apply_H_host",
            "bs_debug_table", "bs_set_kernel", "bs_sync_status", "bs_autotune", "bs_set_tuned", "bs_lanczos",
            "bs_debug_eigh", "bs_apply_H_backward", "bs_block_dots", "bs_block_update", "bs_block_dots_noalloc",
            "bs_debug_eigh_banded", "bs_time_kernel", "bs_kernel_times", "bs_strength", "bs_density", "bs_gather_ceiling",
            "bs_debug_wait_expiry", "bs_build_basis_trunc", "bs_apply_H_host_async"]


class bs_orbit(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("l", ctypes.c_int), ("twoj", ctypes.c_int), ("w", ctypes.c_int)]


class bs_tbme(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int), ("b", ctypes.c_int), ("c", ctypes.c_int), ("d", ctypes.c_int),
                ("J", ctypes.c_int), ("T", ctypes.c_int), ("v", ctypes.c_double)]


class bs_lanczos_opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("dtype", ctypes.c_int), ("niter", ctypes.c_int), ("nkeep", ctypes.c_int),
                ("refine", ctypes.c_int), ("reorth_passes", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("nthick", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("tol", ctypes.c_double), ("targeted", ctypes.c_int), ("target", ctypes.c_double)]


class bs_lanczos_report(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("breakdowns", ctypes.c_int), ("n_kept", ctypes.c_int),
                ("residual", ctypes.c_double * 64), ("delta_conv", ctypes.c_double),
                ("ms_matvec", ctypes.c_double), ("ms_reorth", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("restarts", ctypes.c_int), ("matvec_blocks", ctypes.c_int), ("resid_est", ctypes.c_double)]


class BSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (ERRORS.get(code, "?"), code, msg))
        self.code = code


_lib = None
vp = ctypes.c_void_p
i64p = ctypes.POINTER(ctypes.c_int64)
i32p = ctypes.POINTER(ctypes.c_int)
u64p = ctypes.POINTER(ctypes.c_uint64)
f64p = ctypes.POINTER(ctypes.c_double)


def load():
    """Loads libbsgpu.so; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libbsgpu.so is not built: run paper_1801_08432_gb300.build.build() "
                           "(there is no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    L.bs_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int]
    L.bs_destroy.argtypes = [vp]
    L.bs_destroy.restype = None
    L.bs_last_error.argtypes = [vp]
    L.bs_last_error.restype = ctypes.c_char_p
    L.bs_build_basis.argtypes = [vp, ctypes.POINTER(bs_orbit), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int]
    L.bs_build_basis_trunc.argtypes = [vp, ctypes.POINTER(bs_orbit), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.bs_basis_info.argtypes = [vp, i64p, i32p, i32p, i32p, i32p, i32p]
    L.bs_export_basis.argtypes = [vp, u64p, u64p, i64p, i64p, i64p]
    L.bs_load_interaction.argtypes = [vp, f64p, ctypes.c_int, ctypes.POINTER(bs_tbme), ctypes.c_int]
    L.bs_apply_H.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    L.bs_apply_H_host.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    L.bs_apply_H_host_async.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int]
    L.bs_debug_table.argtypes = [vp, ctypes.c_char_p, vp, i64p]
    L.bs_set_kernel.argtypes = [vp, ctypes.c_int]
    L.bs_set_tuned.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.bs_lanczos.argtypes = [vp, ctypes.POINTER(bs_lanczos_opts), vp, f64p, vp, ctypes.POINTER(bs_lanczos_report)]
    L.bs_strength.argtypes = [vp, ctypes.POINTER(bs_lanczos_opts), vp, ctypes.c_int, f64p, f64p,
                              ctypes.POINTER(bs_lanczos_report)]
    L.bs_density.argtypes = [vp, vp, vp, ctypes.c_int, f64p, vp]
    L.bs_gather_ceiling.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, f64p, vp]
    L.bs_debug_wait_expiry.argtypes = [vp, ctypes.c_int, vp]
    L.bs_debug_eigh.argtypes = [ctypes.c_int, vp, vp, vp, ctypes.c_int]
    L.bs_debug_eigh_banded.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, vp, vp, ctypes.c_int]
    L.bs_apply_H_backward.argtypes = [vp, vp, vp, vp, f64p, ctypes.c_int, ctypes.c_int, vp]
    L.bs_block_dots.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, vp]
    L.bs_block_update.argtypes = [vp, vp, ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int, vp]
    L.bs_block_dots_noalloc.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int, ctypes.c_int, vp, vp]
    L.bs_sync_status.argtypes = [vp, vp]
    L.bs_time_kernel.argtypes = [vp, ctypes.c_int]
    L.bs_kernel_times.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int)]
    L.bs_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_float)]
    for name in EXPORTED:
        if name not in ("bs_destroy", "bs_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _p(a, t):
    return a.ctypes.data_as(t)


class Context:
    """One bs_ctx: a basis, an interaction and their device tables.

    device=-1 builds a host-only context (basis, decoupling and jump tables on
    the CPU, no upload; H*x calls are refused), used to test the host builders
    on machines without a GPU.
    """

    def __init__(self, device: int = 0):
        L = load()
        h = vp()
        rc = L.bs_create(ctypes.byref(h), device)
        if rc != 0:
            raise BSError(rc, "bs_create(device=%d)" % device)
        self.h = h
        self.device = device
        self.dim = None

    def close(self):
        if getattr(self, "h", None):
            load().bs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise BSError(rc, load().bs_last_error(self.h).decode())

    # ---- set-up
    def build_basis(self, orbits, Z, N, twoM, parity=+1, max_excite=None):
        """The M-scheme basis; with max_excite (>= 0) the W-truncated one, the
        orbits' w being the truncation weights."""
        arr = (bs_orbit * len(orbits))(*[bs_orbit(o.n, o.l, o.twoj, o.w) for o in orbits])
        if max_excite is None:
            self._check(load().bs_build_basis(self.h, arr, len(orbits), Z, N, twoM, parity))
        else:
            self._check(load().bs_build_basis_trunc(self.h, arr, len(orbits), Z, N, twoM, parity, max_excite))
        self.info()
        return self

    def info(self):
        dim = ctypes.c_int64()
        v = [ctypes.c_int() for _ in range(5)]
        self._check(load().bs_basis_info(self.h, ctypes.byref(dim), *[ctypes.byref(x) for x in v]))
        self.dim = dim.value
        self.n_psec, self.n_nsec, self.n_psd, self.n_nsd, self.n_blocks = (x.value for x in v)
        return self

    def export_basis(self):
        pb = np.zeros(self.n_psd, dtype=np.uint64)
        nb = np.zeros(self.n_nsd, dtype=np.uint64)
        ps = np.zeros((self.n_psec, 4), dtype=np.int64)
        ns = np.zeros((self.n_nsec, 4), dtype=np.int64)
        bl = np.zeros((self.n_blocks, 3), dtype=np.int64)
        self._check(load().bs_export_basis(self.h, _p(pb, u64p), _p(nb, u64p), _p(ps, i64p), _p(ns, i64p), _p(bl, i64p)))
        return {"p_bits": pb, "n_bits": nb, "p_sec": ps, "n_sec": ns, "blocks": bl}

    def load_interaction(self, spe, tbmes):
        spe = np.ascontiguousarray(spe, dtype=np.float64)
        arr = (bs_tbme * max(1, len(tbmes)))(*[bs_tbme(*t) for t in tbmes])
        self._check(load().bs_load_interaction(self.h, _p(spe, f64p), len(spe), arr, len(tbmes)))
        self.n_spe, self.n_tbme = len(spe), len(tbmes)
        return self

    def table(self, name, dtype):
        n = ctypes.c_int64()
        self._check(load().bs_debug_table(self.h, name.encode(), None, ctypes.byref(n)))
        out = np.zeros(n.value // np.dtype(dtype).itemsize, dtype=dtype)
        self._check(load().bs_debug_table(self.h, name.encode(), out.ctypes.data_as(vp), ctypes.byref(n)))
        return out

    def lanczos(self, pivot, k, dtype, niter, nkeep, refine=True, evecs=None, stream=None, reorth_passes=2,
                use_graph=False, nthick=0, max_restarts=0, tol=0.0, target=None):
        """Block Lanczos on the GPU.  pivot: device tensor [dim][k] (dtype);
        evecs: optional device float64 tensor [dim][nkeep]; nthick > 0 turns
        on thick restart (Ritz vectors kept, a multiple of k) with at most
        max_restarts restarts, stopping once the residual estimates of the
        lowest nkeep pairs are <= tol; target = E_bar runs on (H - E_bar)^2 for
        the levels nearest E_bar.  Returns (eigenvalues as numpy, report
        dict)."""
        o = bs_lanczos_opts(k, dtype, niter, nkeep, int(refine), reorth_passes, int(use_graph), vp(stream or 0),
                            nthick, max_restarts, tol, int(target is not None),
                            0.0 if target is None else float(target))
        ev = np.zeros(nkeep)
        rep = bs_lanczos_report()
        pp = pivot if isinstance(pivot, int) else pivot.data_ptr()
        ep = None if evecs is None else vp(evecs if isinstance(evecs, int) else evecs.data_ptr())
        self._check(load().bs_lanczos(self.h, ctypes.byref(o), vp(pp), ev.ctypes.data_as(f64p), ep, ctypes.byref(rep)))
        r = {"iterations": rep.iterations, "breakdowns": rep.breakdowns, "n_kept": rep.n_kept,
             "residual": [rep.residual[i] for i in range(rep.n_kept)], "delta_conv": rep.delta_conv,
             "ms_matvec": rep.ms_matvec, "ms_reorth": rep.ms_reorth, "ms_total": rep.ms_total,
             "restarts": rep.restarts, "matvec_blocks": rep.matvec_blocks, "resid_est": rep.resid_est}
        return ev, r

    def strength(self, pivot, k, dtype, niter, n_out, stream=None, use_graph=False, reorth_passes=2):
        """Strength function from the pivot block (device tensor [dim][k], any
        norm): (E [n_out], S [k][n_out]) as numpy, S = |<w_i|E_r>|^2, plus the
        report dict."""
        o = bs_lanczos_opts(k, dtype, niter, 1, 0, reorth_passes, int(use_graph), vp(stream or 0), 0, 0, 0.0, 0, 0.0)
        E = np.zeros(n_out)
        S = np.zeros((k, n_out))
        rep = bs_lanczos_report()
        pp = pivot if isinstance(pivot, int) else pivot.data_ptr()
        self._check(load().bs_strength(self.h, ctypes.byref(o), vp(pp), n_out, E.ctypes.data_as(f64p),
                                       S.ctypes.data_as(f64p), ctypes.byref(rep)))
        return E, S, {"iterations": rep.iterations, "breakdowns": rep.breakdowns, "ms_total": rep.ms_total,
                      "ms_matvec": rep.ms_matvec, "ms_reorth": rep.ms_reorth}

    def density(self, F, X, k, ns, stream=None):
        """One-body transition densities rho[t][i][l][f][j] = <F_f| a+_i a_l |X_j>
        (numpy, t = 0 protons, 1 neutrons) of the k columns of two FP64 CUDA
        tensors [dim][k] on this basis; ns single-particle states."""
        rho = np.zeros((2, ns, ns, k, k))
        ptr = lambda t: vp(t if isinstance(t, int) else t.data_ptr())
        self._check(load().bs_density(self.h, ptr(F), ptr(X), k, rho.ctypes.data_as(f64p), vp(stream or 0)))
        return rho

    def gather_ceiling(self, where, k, rows, stream=None):
        """Measured GFLOP/s of the gather + FMA step (where 0: shared memory,
        1: L2), k-float elements applied to `rows` accumulator rows."""
        g = ctypes.c_double(0.0)
        self._check(load().bs_gather_ceiling(self.h, where, k, rows, ctypes.byref(g), vp(stream or 0)))
        return g.value

    def set_kernel(self, mode):
        self._check(load().bs_set_kernel(self.h, mode))

    def autotune(self, k, dtype, stream=None, times=False):
        """Picks the fastest kernel mode for (k, dtype); with times=True also
        returns {mode: ms per product}."""
        m = ctypes.c_int()
        ms = (ctypes.c_float * KERNEL_MODES)()
        self._check(load().bs_autotune(self.h, k, dtype, vp(stream or 0), ctypes.byref(m), ms))
        if times:
            return m.value, {i + 1: round(float(ms[i]), 4) for i in range(KERNEL_MODES)}
        return m.value

    def set_tuned(self, k, dtype, mode):
        """Record `mode` as the autotuned kernel mode for (k, dtype) (no timing)."""
        self._check(load().bs_set_tuned(self.h, k, dtype, mode))

    def time_kernel(self, n):
        """Record CUDA events around the dominant kernel of the next n products."""
        self._check(load().bs_time_kernel(self.h, n))

    def kernel_times(self):
        """Milliseconds of the recorded launches (waits for them)."""
        n = ctypes.c_int()
        self._check(load().bs_kernel_times(self.h, None, ctypes.byref(n)))
        ms = np.zeros(max(n.value, 1), dtype=np.float32)
        self._check(load().bs_kernel_times(self.h, ms.ctypes.data_as(vp), ctypes.byref(n)))
        return ms[:n.value]

    def sync_status(self, stream=None):
        self._check(load().bs_sync_status(self.h, vp(stream or 0)))

    # ---- products
    def apply_H(self, x, y, k, dtype, stream=None):
        """y = H x; x, y: torch CUDA tensors [dim][k] (or raw device pointers)."""
        xp = x if isinstance(x, int) else x.data_ptr()
        yp = y if isinstance(y, int) else y.data_ptr()
        self._check(load().bs_apply_H(self.h, vp(xp), vp(yp), k, dtype, vp(stream or 0)))

    def apply_H_backward(self, x, gy, gx, k, dtype, n_theta=None, stream=None):
        """gx = H gy; returns gtheta (numpy, n_spe + n_tbme) = sum gy^T dH/dtheta x,
        or None when n_theta is None."""
        ptr = lambda t: vp(t if isinstance(t, int) else t.data_ptr())
        g = None if n_theta is None else np.zeros(n_theta)
        self._check(load().bs_apply_H_backward(self.h, ptr(x), ptr(gy), ptr(gx),
                                               None if g is None else g.ctypes.data_as(f64p), k, dtype,
                                               vp(stream or 0)))
        return g

    def block_dots(self, V, nb, W, k, dtype, C, stream=None):
        """C[b][i][j] = sum_alpha V_b[alpha][i] W[alpha][j]; V, W, C device tensors
        (C float64 with nb*k*k elements)."""
        ptr = lambda t: vp(t if isinstance(t, int) else t.data_ptr())
        self._check(load().bs_block_dots(self.h, ptr(V), nb, ptr(W), k, dtype, ptr(C), vp(stream or 0)))

    def block_update(self, V, nb, C, W, k, dtype, stream=None):
        """W -= sum_b V_b C_b; V, C (float64, nb*k*k), W device tensors."""
        ptr = lambda t: vp(t if isinstance(t, int) else t.data_ptr())
        self._check(load().bs_block_update(self.h, ptr(V), nb, ptr(C), ptr(W), k, dtype, vp(stream or 0)))

    def apply_H_host(self, x, y, k, dtype, stream=None):
        """y = H x with host numpy buffers (copies inside)."""
        self._check(load().bs_apply_H_host(self.h, x.ctypes.data_as(vp), y.ctypes.data_as(vp), k, dtype,
                                           vp(stream or 0)))

    def apply_H_host_async(self, x, y, k, dtype, stream, slot):
        """y = H x with pinned host buffers (torch tensors, numpy arrays or raw
        addresses), enqueued on `stream` in staging slot 0 or 1 without waiting;
        synchronize the stream before reading y or rewriting x."""
        def ptr(t):
            if isinstance(t, int):
                return vp(t)
            return vp(t.data_ptr()) if hasattr(t, "data_ptr") else t.ctypes.data_as(vp)
        self._check(load().bs_apply_H_host_async(self.h, ptr(x), ptr(y), k, dtype, vp(stream or 0), slot))


def make(space_orbits, spe, tbmes, Z, N, twoM, parity=+1, device=0, max_excite=None):
    return Context(device).build_basis(space_orbits, Z, N, twoM, parity, max_excite).load_interaction(spe, tbmes)


def debug_eigh(A, nvec):
    """The library's host FP64 symmetric eigensolver (test aid)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(n)
    Z = np.zeros((n, max(nvec, 1)))
    rc = load().bs_debug_eigh(n, A.ctypes.data_as(vp), w.ctypes.data_as(vp), Z.ctypes.data_as(vp), nvec)
    if rc != 0:
        raise BSError(rc, "bs_debug_eigh")
    return w, Z[:, :nvec]


def debug_eigh_banded(A, bw, nval, nvec):
    """The library's banded host FP64 eigensolver (test aid)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    w = np.zeros(max(nval, 1))
    Z = np.zeros((n, max(nvec, 1)))
    rc = load().bs_debug_eigh_banded(n, bw, A.ctypes.data_as(vp), nval, w.ctypes.data_as(vp), Z.ctypes.data_as(vp), nvec)
    if rc != 0:
        raise BSError(rc, "bs_debug_eigh_banded")
    return w[:nval], Z[:, :nvec]
