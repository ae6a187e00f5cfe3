"""FP64 CPU oracle for the factorized M-scheme H*x (BIGSTICK, arXiv:1801.08432).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  It shares no code with the
library in ``paper_1801_08432_gb300`` and never imports it (apart from the
seeded input generators in ``paper_1801_08432_gb300.inputs``, which hold none
of the method's arithmetic).

Parts:
  * ``bs_oracle.c`` (plain C, FP64): basis of occupation bitstrings, the
    Clebsch-Gordan coefficient, reading of isospin-coupled TBMEs with their
    symmetry phases, decoupling to M-scheme W tables, the explicit Hamiltonian
    built column by column from creation/annihilation operators, on-the-fly
    rows of H*x and J+.
  * this module (numpy/scipy): Lanczos with full reorthogonalization (Sec.
    "Standard Lanczos algorithm", steps (1)-(6) with alpha computed first and
    then orthogonalization against every earlier vector); thick-restart block
    Lanczos, plain and targeted at interior levels; the block strength
    function; dense diagonalization; <J^2>; orbit occupations; M-scheme and
    reduced one-body densities; the W-truncated Hamiltonian; traces and
    Hellmann-Feynman gradients.

Parity pins: every function here is checked in tests/test_oracle_pins.py
against closed forms, paper values or brute force (see that file's header).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

i64p = ctypes.POINTER(ctypes.c_int64)
u64p = ctypes.POINTER(ctypes.c_uint64)
f64p = ctypes.POINTER(ctypes.c_double)
i32p = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compiles bs_oracle.c into liboracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            L.orc_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), i32p, i32p, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            L.orc_create.restype = ctypes.c_int
            L.orc_dim.argtypes = [ctypes.c_void_p]
            L.orc_dim.restype = ctypes.c_int64
            L.orc_ns.argtypes = [ctypes.c_void_p]
            L.orc_ns.restype = ctypes.c_int
            L.orc_sizes.argtypes = [ctypes.c_void_p, i32p]
            L.orc_export_basis.argtypes = [ctypes.c_void_p, u64p, u64p, i64p, i64p, i64p]
            L.orc_set_interaction.argtypes = [ctypes.c_void_p, f64p, i32p, f64p, ctypes.c_int]
            L.orc_set_interaction.restype = ctypes.c_int
            L.orc_get_w.argtypes = [ctypes.c_void_p, f64p, f64p]
            L.orc_build_matrix.argtypes = [ctypes.c_void_p]
            L.orc_build_matrix.restype = ctypes.c_int64
            L.orc_export_matrix.argtypes = [ctypes.c_void_p, i64p, i64p, f64p]
            L.orc_spmv.argtypes = [ctypes.c_void_p, f64p, f64p, ctypes.c_int]
            L.orc_build_rows.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int64]
            L.orc_build_rows.restype = ctypes.c_int64
            L.orc_spmv_rows.argtypes = [ctypes.c_void_p, f64p, f64p, ctypes.c_int]
            L.orc_apply_rows.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int64, f64p, ctypes.c_int, f64p]
            L.orc_apply_rows_ex.argtypes = [ctypes.c_void_p, i64p, ctypes.c_int64, f64p, ctypes.c_int, f64p, ctypes.c_int]
            L.orc_jplus.argtypes = [ctypes.c_void_p, ctypes.c_void_p, f64p, f64p]
            L.orc_jplus.restype = ctypes.c_int
            L.orc_cg.argtypes = [ctypes.c_int] * 6
            L.orc_cg.restype = ctypes.c_double
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_apply_string.argtypes = [ctypes.c_uint64, i32p, ctypes.c_int, u64p]
            L.orc_apply_string.restype = ctypes.c_int
            _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def cg(tj1, tm1, tj2, tm2, tJ, tM) -> float:
    """<j1 m1 j2 m2 | J M> (Edmonds), all arguments doubled."""
    return lib().orc_cg(tj1, tm1, tj2, tm2, tJ, tM)


def apply_string(mask: int, ops):
    """Sign and result of an operator string on a bitstring (bit s = state s).

    ops is a list of ('+', s) for a^dag_s or ('-', s) for a_s, written left
    to right as in the paper; the rightmost acts first.  Returns (sign, mask),
    sign 0 if the state vanishes."""
    enc = np.array([(s + 1) if c == "+" else -(s + 1) for (c, s) in ops], dtype=np.int32)
    out = ctypes.c_uint64(0)
    sg = lib().orc_apply_string(ctypes.c_uint64(mask), _p(enc, i32p), len(enc), ctypes.byref(out))
    return sg, (out.value if sg else None)


class OracleError(RuntimeError):
    pass


class Oracle:
    """One valence space, one nucleus (Z, N), one 2M and parity (0 = +, 1 = -)."""

    def __init__(self, orbits, Z, N, twoM, parity=0):
        L = lib()
        self.orbits = list(orbits)
        l = np.array([o.l for o in orbits], dtype=np.int32)
        tj = np.array([o.twoj for o in orbits], dtype=np.int32)
        h = ctypes.c_void_p()
        rc = L.orc_create(ctypes.byref(h), _p(l, i32p), _p(tj, i32p), len(orbits), Z, N, twoM, parity)
        if rc != 0:
            raise OracleError("orc_create failed (%d)" % rc)
        self.h = h
        self.Z, self.N, self.twoM, self.parity = Z, N, twoM, parity
        self.dim = int(L.orc_dim(h))
        self.ns = int(L.orc_ns(h))
        sz = np.zeros(5, dtype=np.int32)
        L.orc_sizes(h, _p(sz, i32p))
        self.n_psd, self.n_nsd, self.n_psec, self.n_nsec, self.n_blocks = (int(v) for v in sz)
        self._csr = None
        self._nnz = None

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().orc_destroy(self.h)
                self.h = None
        except Exception:
            pass

    # -- basis -----------------------------------------------------------
    def basis(self):
        """dict: p_bits, n_bits (uint64), p_sec/n_sec rows (2M, par, start, count),
        blocks rows (proton sector, neutron sector, offset)."""
        pb = np.zeros(self.n_psd, dtype=np.uint64)
        nb = np.zeros(self.n_nsd, dtype=np.uint64)
        ps = np.zeros((self.n_psec, 4), dtype=np.int64)
        nsec = np.zeros((self.n_nsec, 4), dtype=np.int64)
        bl = np.zeros((self.n_blocks, 3), dtype=np.int64)
        lib().orc_export_basis(self.h, _p(pb, u64p), _p(nb, u64p), _p(ps, i64p), _p(nsec, i64p), _p(bl, i64p))
        return {"p_bits": pb, "n_bits": nb, "p_sec": ps, "n_sec": nsec, "blocks": bl}

    def states(self):
        """(basis index) -> (proton bits, neutron bits) for every basis state, as two arrays."""
        B = self.basis()
        P = np.zeros(self.dim, dtype=np.uint64)
        Nn = np.zeros(self.dim, dtype=np.uint64)
        for (ps, nsi, off) in B["blocks"]:
            _, _, p0, pc = B["p_sec"][ps]
            _, _, n0, nc = B["n_sec"][nsi]
            pbits = B["p_bits"][p0:p0 + pc]
            nbits = B["n_bits"][n0:n0 + nc]
            P[off:off + pc * nc] = np.repeat(pbits, nc)
            Nn[off:off + pc * nc] = np.tile(nbits, pc)
        return P, Nn

    # -- interaction -----------------------------------------------------
    def set_interaction(self, spe, tbmes):
        spe = np.ascontiguousarray(spe, dtype=np.float64)
        lab = np.array([t[:6] for t in tbmes], dtype=np.int32).reshape(-1, 6)
        val = np.array([t[6] for t in tbmes], dtype=np.float64)
        rc = lib().orc_set_interaction(self.h, _p(spe, f64p), _p(lab, i32p), _p(val, f64p), len(tbmes))
        if rc != 0:
            raise OracleError("orc_set_interaction rejected the interaction (%d)" % rc)
        self._csr = None
        self._nnz = None
        return self

    def w_tables(self):
        n4 = self.ns ** 4
        wpp = np.zeros(n4)
        wpn = np.zeros(n4)
        lib().orc_get_w(self.h, _p(wpp, f64p), _p(wpn, f64p))
        s = (self.ns,) * 4
        return wpp.reshape(s), wpn.reshape(s)

    # -- Hamiltonian -----------------------------------------------------
    def build_matrix(self):
        """Builds the explicit H in the C part (its columns, which are its rows
        since H = H^T) and returns the number of stored elements.  spmv() needs
        only this; matrix() also copies it out to scipy."""
        if self._nnz is None:
            nnz = lib().orc_build_matrix(self.h)
            if nnz < 0:
                raise OracleError("orc_build_matrix failed (%d)" % nnz)
            self._nnz = int(nnz)
        return self._nnz

    def matrix(self):
        """Explicit H as scipy.sparse.csr_matrix (FP64)."""
        import scipy.sparse as sp
        if self._csr is None:
            nnz = self.build_matrix()
            cp = np.zeros(self.dim + 1, dtype=np.int64)
            ri = np.zeros(max(nnz, 1), dtype=np.int64)
            va = np.zeros(max(nnz, 1))
            lib().orc_export_matrix(self.h, _p(cp, i64p), _p(ri, i64p), _p(va, f64p))
            # stored columns of H; csc -> csr through the transpose
            self._csr = sp.csc_matrix((va[:nnz], ri[:nnz], cp), shape=(self.dim, self.dim)).tocsr()
        return self._csr

    def spmv(self, x):
        """y = H x with the explicit matrix, x [dim] or [dim][k] (the C part's
        stored rows, OpenMP over rows)."""
        self.build_matrix()
        x = np.ascontiguousarray(x, dtype=np.float64)
        k = 1 if x.ndim == 1 else x.shape[1]
        y = np.zeros_like(x)
        lib().orc_spmv(self.h, _p(x, f64p), _p(y, f64p), k)
        return y

    def build_rows(self, rows):
        """Stores the given rows of the explicit H (built as build_matrix()
        builds every row) for spmv_rows(); returns their element count."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        nnz = lib().orc_build_rows(self.h, _p(rows, i64p), len(rows))
        if nnz < 0:
            raise OracleError("orc_build_rows failed (%d)" % nnz)
        self._sub_rows = rows
        return int(nnz)

    def spmv_rows(self, x):
        """The rows stored by build_rows() of y = H x, x [dim] or [dim][k]:
        the stored-matrix product (spmv) restricted to a sample of rows."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        k = 1 if x.ndim == 1 else x.shape[1]
        y = np.zeros((len(self._sub_rows), k))
        lib().orc_spmv_rows(self.h, _p(x, f64p), _p(y, f64p), k)
        return y[:, 0] if x.ndim == 1 else y

    def apply_rows(self, rows, x, absval=False):
        """Rows of y = H x computed on the fly (no stored matrix); with
        absval=True rows of |H| |x| (a bound for rounding errors)."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        k = 1 if x.ndim == 1 else x.shape[1]
        y = np.zeros((len(rows), k))
        lib().orc_apply_rows_ex(self.h, _p(rows, i64p), len(rows), _p(x, f64p), k, _p(y, f64p), int(absval))
        return y[:, 0] if x.ndim == 1 else y

    def dense(self):
        return self.matrix().toarray()

    def trace(self):
        return float(self.matrix().diagonal().sum())

    # -- eigen -----------------------------------------------------------
    def lanczos(self, pivot, niter, nkeep=None, return_vectors=False):
        """Lanczos with full reorthogonalization (FP64).

        Per iteration: w = H v_i; alpha_i = <v_i|w>; w -= alpha_i v_i; then
        w -= v_j <v_j|w> for every j <= i, twice (classical Gram-Schmidt);
        beta_i = |w|; v_{i+1} = w / beta_i.  Eigenvalues of the tridiagonal
        matrix by numpy.linalg.eigh; Ritz vectors from its eigenvectors.
        H v is the explicit matrix's product (spmv), so a space as large as
        pf 4p4n needs only the C part's copy of H.
        """
        v = np.array(pivot, dtype=np.float64).reshape(-1)
        v = v / np.linalg.norm(v)
        niter = min(niter, self.dim)
        V = np.zeros((niter, self.dim))
        alpha = np.zeros(niter)
        beta = np.zeros(niter)
        n = 0
        for i in range(niter):
            V[i] = v
            w = self.spmv(v)
            alpha[i] = v @ w
            w = w - alpha[i] * v
            for _ in range(2):
                w = w - V[: i + 1].T @ (V[: i + 1] @ w)
            n = i + 1
            beta[i] = np.linalg.norm(w)
            if i + 1 == niter or beta[i] < 1e-12 * max(1.0, np.abs(alpha[: i + 1]).max()):
                break
            v = w / beta[i]
        T = np.diag(alpha[:n]) + np.diag(beta[: n - 1], 1) + np.diag(beta[: n - 1], -1)
        ev, U = np.linalg.eigh(T)
        if not return_vectors:
            return ev if nkeep is None else ev[:nkeep]
        nk = n if nkeep is None else nkeep
        X = V[:n].T @ U[:, :nk]
        return ev[:nk], X

    def block_lanczos_thick(self, pivot, niter, nthick, restarts, nkeep=None, return_vectors=False,
                            return_state=False, target=None):
        """Thick-restart block Lanczos (FP64): Sec. "Block Lanczos", Sec.
        "Thick-restart Lanczos" and Sec. "Thick-restart block Lanczos".

        pivot: [dim][k] block.  One cycle builds blocks V_n, n0 <= n < niter,
        each with  W = H V_n;  A_n = V_n^T W;  W -= V_n A_n;  then twice
        W -= Q (Q^T W) over every stored block Q;  O = W^T W = U L U^T;
        B_n = L^(1/2) U^T;  V_(n+1) = W U L^(-1/2).  T (niter k square) holds
        A_n on the diagonal and B_n below it.  After a restart its leading
        nthick x nthick part is the diagonal of the kept Ritz values E and
        the block row of V_t (t = nthick / k, the restart pivot) holds
        r = B_last U[last block rows, :nthick] against them (the arrow of the
        thick-restart matrix).  A restart diagonalizes T, keeps the lowest
        nthick Ritz vectors Q U[:, :nthick] as the first t blocks, and takes
        the last Lanczos block V_niter as V_t.  ``restarts`` restarts are
        done, so restarts + 1 cycles.

        Returns the eigenvalues of the last T (the lowest nkeep, or all) and
        per cycle the list of all Ritz values; with ``return_vectors`` also
        the Ritz vectors of the lowest nkeep; with ``return_state`` also the
        last cycle's stored blocks Q ([dim][niter k]) and T.

        ``target`` = E_bar runs the same iteration on (H - E_bar)^2
        (Sec. "Targeted thick-restart Lanczos: interior eigenvalues"): the
        levels nearest E_bar become the lowest of that operator, and T holds
        its projection.
        """
        H0 = self.matrix()
        if target is None:
            H = H0
        else:
            class _Shifted2:   # v -> (H - E_bar)^2 v
                def __matmul__(_, v):
                    w = H0 @ v - target * v
                    return H0 @ w - target * w
            H = _Shifted2()
        X = np.array(pivot, dtype=np.float64).reshape(self.dim, -1)
        k = X.shape[1]
        if nthick % k or not 0 <= nthick // k < niter - 1:
            raise ValueError("nthick must be a multiple of k with nthick / k + 1 < niter")
        t = nthick // k

        def orthonormal(W):
            lam, U = np.linalg.eigh(W.T @ W)
            if lam[0] <= 1e-24 * lam[-1]:
                raise OracleError("block Lanczos breakdown")
            return W @ (U / np.sqrt(lam)), (np.sqrt(lam)[:, None] * U.T)

        Q = [orthonormal(X)[0]]
        E = R = None
        history = []
        for cycle in range(restarts + 1):
            n0 = 0 if cycle == 0 else t
            A, B = {}, {}
            for n in range(n0, niter):
                W = H @ Q[n]
                A[n] = Q[n].T @ W
                W = W - Q[n] @ A[n]
                S = np.hstack(Q)
                for _ in range(2):
                    W = W - S @ (S.T @ W)
                Vn1, B[n] = orthonormal(W)
                Q.append(Vn1)
            nT = niter * k
            T = np.zeros((nT, nT))
            if cycle > 0:
                T[:nthick, :nthick] = np.diag(E)
                T[t * k:(t + 1) * k, :nthick] = R
                T[:nthick, t * k:(t + 1) * k] = R.T
            for n in range(n0, niter):
                T[n * k:(n + 1) * k, n * k:(n + 1) * k] = 0.5 * (A[n] + A[n].T)
                if n + 1 < niter:
                    T[(n + 1) * k:(n + 2) * k, n * k:(n + 1) * k] = B[n]
                    T[n * k:(n + 1) * k, (n + 1) * k:(n + 2) * k] = B[n].T
            ev, Z = np.linalg.eigh(T)
            history.append(ev.copy())
            if cycle == restarts:
                break
            S = np.hstack(Q[:niter])
            Y = S @ Z[:, :nthick]
            R = B[niter - 1] @ Z[(niter - 1) * k:niter * k, :nthick]
            E = ev[:nthick]
            Q = [Y[:, j * k:(j + 1) * k] for j in range(t)] + [Q[niter]]
        nk = len(ev) if nkeep is None else nkeep
        out = [ev[:nk], history]
        if return_vectors:
            out.append(np.hstack(Q[:niter]) @ Z[:, :nk])
        if return_state:
            out += [np.hstack(Q[:niter]), T]
        return tuple(out)

    def strength(self, pivot, niter):
        """Block strength function (FP64): Sec. "Generating strength function
        distributions" and Sec. "Block strength function".

        pivot: [dim][k] block W_0 of any norm.  Its overlap matrix
        O = W_0^T W_0 = U L U^T gives the orthonormal pivot V_1 = W_0 U L^(-1/2)
        and B_0 = L^(1/2) U^T (so W_0 = V_1 B_0); niter block Lanczos
        iterations with full reorthogonalization follow (as in
        ``block_lanczos_thick`` without restart).  With T = L_T E L_T^T the
        overlaps are <w_i|E_r> = sum_j (B_0)_ji (L_T)_jr over the first block's
        rows j.  Returns (E [n], S [k][n]) with S = |<w_i|E_r>|^2 for every
        eigenvalue of T (n = niter k)."""
        W0 = np.array(pivot, dtype=np.float64).reshape(self.dim, -1)
        k = W0.shape[1]
        lam, U = np.linalg.eigh(W0.T @ W0)
        if lam[0] <= 1e-24 * lam[-1]:
            raise OracleError("rank-deficient pivot block")
        B0 = np.sqrt(lam)[:, None] * U.T
        V1 = W0 @ (U / np.sqrt(lam))
        H = self.matrix()
        Q = [V1]
        A, B = [], []
        for n in range(niter):
            W = H @ Q[n]
            A.append(Q[n].T @ W)
            W = W - Q[n] @ A[n]
            S = np.hstack(Q)
            for _ in range(2):
                W = W - S @ (S.T @ W)
            l2, U2 = np.linalg.eigh(W.T @ W)
            if l2[0] <= 1e-24 * max(l2[-1], 1e-300):
                raise OracleError("block Lanczos breakdown")
            B.append(np.sqrt(l2)[:, None] * U2.T)
            Q.append(W @ (U2 / np.sqrt(l2)))
        nT = niter * k
        T = np.zeros((nT, nT))
        for n in range(niter):
            T[n * k:(n + 1) * k, n * k:(n + 1) * k] = 0.5 * (A[n] + A[n].T)
            if n + 1 < niter:
                T[(n + 1) * k:(n + 2) * k, n * k:(n + 1) * k] = B[n]
                T[n * k:(n + 1) * k, (n + 1) * k:(n + 2) * k] = B[n].T
        E, LT = np.linalg.eigh(T)
        ov = B0.T @ LT[:k, :]
        return E, ov * ov

    def eigh(self, nkeep=None):
        ev, X = np.linalg.eigh(self.dense())
        if nkeep is None:
            return ev, X
        return ev[:nkeep], X[:, :nkeep]

    # -- occupations -----------------------------------------------------
    def occupations(self, psi):
        """n_a = sum_alpha psi_alpha^2 (protons + neutrons of SD alpha in
        orbit a) / |psi|^2, per orbit a (Sec. "Occupations": the number of
        nucleons in each orbit).  Single-particle states are numbered
        orbit-major, 2m ascending, so orbit a owns a run of 2j_a + 1 bits."""
        psi = np.asarray(psi, dtype=np.float64)
        w = psi * psi / float(psi @ psi)
        P, Nn = self.states()
        ones = np.array([bin(v).count("1") for v in range(256)], dtype=np.int64)

        def popcount(x):
            return ones[x.view(np.uint8).reshape(-1, 8)].sum(axis=1)

        out, off = [], 0
        for o in self.orbits:
            mask = np.uint64(((1 << (o.twoj + 1)) - 1) << off)
            out.append(float(w @ (popcount(P & mask) + popcount(Nn & mask))))
            off += o.twoj + 1
        return np.array(out)

    def isospin_density(self, red, twoTf, twoTi):
        """Doubly reduced (J and isospin) one-body densities from the reduced
        proton-neutron ones ``red`` (as returned by ``reduced_density``), for
        states of good isospin T_f, T_i (Sec. "Conversion from proton-neutron
        to isospin"; protons m_t = +1/2, T_z = (Z - N)/2):

            rho_T = [T_f] / (T_i T_z, T 0 | T_f T_z) [T]^-1
                    sum_{m_t} (-1)^(1/2 - m_t) (1/2 m_t, 1/2 -m_t | T 0) rho_{m_t}

        with the isospin time-reversal phase of c~ written out.  Returns
        {(a, b, 2K, T): value}, NaN where the isospin coefficient vanishes."""
        tTz = self.Z - self.N
        out = {}
        keys = {(a, b, tk) for (t, a, b, tk) in red}
        for (a, b, tk) in keys:
            for T in (0, 1):
                c = cg(twoTi, tTz, 2 * T, 0, twoTf, tTz)
                if abs(c) < 1e-12:
                    out[(a, b, tk, T)] = np.nan
                    continue
                acc = 0.0
                for t, tmt in ((0, 1), (1, -1)):   # protons m_t = +1/2, neutrons -1/2
                    ph = 1.0 if t == 0 else -1.0   # (-1)^(1/2 - m_t)
                    acc += ph * cg(1, tmt, 1, -tmt, 2 * T, 0) * red[(t, a, b, tk)]
                out[(a, b, tk, T)] = np.sqrt(twoTf + 1.0) / c / np.sqrt(2 * T + 1.0) * acc
        return out

    # -- W truncation -----------------------------------------------------
    def truncation_mask(self, weights, max_excite):
        """Basis states kept by the W truncation (Sec. "Truncation of the
        many-body space"): every orbit a carries a non-negative integer w_a,
        a state's W is the sum of w over its occupied proton and neutron
        states, W_min is the smallest W any Z-proton, N-neutron state can
        have (the lowest-w states filled), and the kept states have
        W <= W_min + max_excite.  Returns (mask over this basis, W_min,
        largest possible excitation)."""
        st = self.sp_states()
        w_state = np.array([weights[a] for (a, _) in st], dtype=np.int64)
        srt = np.sort(w_state)
        w_min = int(srt[:self.Z].sum() + srt[:self.N].sum())
        w_max = int(srt[::-1][:self.Z].sum() + srt[::-1][:self.N].sum())
        P, Nn = self.states()
        W = np.zeros(self.dim, dtype=np.int64)
        for s_idx in range(self.ns):
            bit = np.uint64(1) << np.uint64(s_idx)
            W += w_state[s_idx] * (((P & bit) != 0).astype(np.int64) + ((Nn & bit) != 0).astype(np.int64))
        return W <= w_min + max_excite, w_min, w_max - w_min

    def truncated_matrix(self, weights, max_excite):
        """The Hamiltonian of the truncated space: H restricted to the kept
        basis states (rows and columns), in their basis order."""
        mask, _, _ = self.truncation_mask(weights, max_excite)
        idx = np.nonzero(mask)[0]
        return self.matrix()[idx][:, idx]

    # -- one-body densities ----------------------------------------------
    def sp_states(self):
        """(orbit, 2m) of every single-particle state: orbit-major, 2m ascending."""
        out = []
        for a, o in enumerate(self.orbits):
            out += [(a, tm) for tm in range(-o.twoj, o.twoj + 1, 2)]
        return out

    def density(self, F, X, other=None):
        """M-scheme one-body transition densities (Sec. "One-body density
        matrices and occupations", before the reduction):

            rho[t][i][k] = <F| a+_i a_k |X>   (t = 0 protons, 1 neutrons)

        for vectors X in this basis and F in ``other``'s (default: this one),
        every single-particle pair (i, k).  Each term applies a_k and then
        a+_i to the species' bitstring with the sign (-1)^(number of occupied
        states below the acted-on state), finds the resulting state in F's
        basis and adds sign F[dst] X[src]; a pair of operators of one species
        passes the other species' operators without a sign."""
        fo = self if other is None else other
        X = np.asarray(X, dtype=np.float64)
        F = np.asarray(F, dtype=np.float64)
        ns = self.ns
        P, Nn = self.states()
        Pf, Nf = fo.states()
        key_f = (Pf << np.uint64(ns)) | Nf
        order = np.argsort(key_f)
        sorted_f = key_f[order]
        ones = np.array([bin(v).count("1") for v in range(256)], dtype=np.int64)

        def popcount(x):
            return ones[x.view(np.uint8).reshape(-1, 8)].sum(axis=1)

        st = self.sp_states()
        dtm = fo.twoM - self.twoM
        rho = np.zeros((2, ns, ns))
        for t in range(2):
            bits = P if t == 0 else Nn
            for i in range(ns):
                for k in range(ns):
                    if st[i][1] - st[k][1] != dtm or self.orbits[st[i][0]].l % 2 != self.orbits[st[k][0]].l % 2:
                        continue
                    bk, bi = np.uint64(1) << np.uint64(k), np.uint64(1) << np.uint64(i)
                    ok = (bits & bk) != 0
                    b1 = bits ^ bk
                    ok &= (b1 & bi) == 0
                    if not ok.any():
                        continue
                    idx = np.nonzero(ok)[0]
                    below_k = popcount(bits[idx] & (bk - np.uint64(1)))
                    b1 = b1[idx]
                    below_i = popcount(b1 & (bi - np.uint64(1)))
                    b2 = b1 | bi
                    sign = np.where((below_k + below_i) % 2 == 0, 1.0, -1.0)
                    key = (b2 << np.uint64(ns)) | Nn[idx] if t == 0 else (P[idx] << np.uint64(ns)) | b2
                    pos = np.searchsorted(sorted_f, key)
                    pos = np.minimum(pos, len(sorted_f) - 1)
                    hit = sorted_f[pos] == key
                    dst = order[pos[hit]]
                    rho[t, i, k] = float(np.sum(sign[hit] * F[dst] * X[idx[hit]]))
        return rho

    def reduced_density(self, rho, twoJf, twoJi):
        """Reduced one-body densities in proton-neutron form (Sec. "One-body
        density matrices and occupations"), from the M-scheme densities
        ``rho`` (as returned by ``density`` for two states of this basis,
        M_f = M_i = M):

            rho_K(a+ b) = [K]^-1 <J_f||(a+ b~)_K||J_i>,
            (a+ b~)_K0 = sum_m (j_a m, j_b -m | K 0) a+_{a m} b~_{b -m},
            b~_{b -m} = (-1)^(j_b - m) b_{b m},
            <J_f||O_K||J_i> = [J_f] <J_f M|O_K0|J_i M> / (J_i M, K 0 | J_f M)

        with [x] = sqrt(2x + 1) and Edmonds' Wigner-Eckart convention.
        Returns {(t, a, b, 2K): value}, NaN where the Clebsch-Gordan
        coefficient vanishes at this M."""
        st = self.sp_states()
        tM = self.twoM
        out = {}
        na = len(self.orbits)
        for t in range(2):
            for a in range(na):
                for b in range(na):
                    ja, jb = self.orbits[a].twoj, self.orbits[b].twoj
                    for twoK in range(abs(ja - jb), ja + jb + 1, 2):
                        s = 0.0
                        for i, (oa, tma) in enumerate(st):
                            if oa != a:
                                continue
                            for l, (ob, tmb) in enumerate(st):
                                if ob == b and tmb == tma:
                                    ph = -1.0 if ((jb - tma) // 2) % 2 else 1.0
                                    s += cg(ja, tma, jb, -tma, twoK, 0) * ph * rho[t, i, l]
                        c = cg(twoJi, tM, twoK, 0, twoJf, tM)
                        out[(t, a, b, twoK)] = (np.nan if abs(c) < 1e-12 else
                                                np.sqrt(twoJf + 1.0) * s / c / np.sqrt(twoK + 1.0))
        return out

    # -- J^2 ------------------------------------------------------------
    def j2(self, psi, oracle_up):
        """<J^2> = |J+ psi|^2 + M(M+1), with J+ psi evaluated in the 2M+2 basis."""
        psi = np.ascontiguousarray(psi, dtype=np.float64)
        out = np.zeros(oracle_up.dim)
        rc = lib().orc_jplus(self.h, oracle_up.h, _p(psi, f64p), _p(out, f64p))
        if rc != 0:
            raise OracleError("orc_jplus failed")
        M = self.twoM / 2.0
        return float(out @ out) / float(psi @ psi) + M * (M + 1.0)


def j_from_j2(j2):
    """J from J(J+1)."""
    return 0.5 * (-1.0 + np.sqrt(1.0 + 4.0 * np.asarray(j2)))
