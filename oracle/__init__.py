"""FP64 CPU oracle for cluster-TEBD (arXiv 2502.19289) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The
product library (``paper_2502_19289_gb300``) never imports, links or runs it,
and this package imports nothing from the product.

The arithmetic lives in ``oracle.c`` (plain C99 + complex.h, double
precision, single-threaded).  This module compiles it with gcc on first use
and wraps it with ctypes.  Every function states the passage it follows.

Parity status: every function below is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, App. A, the brute-force
state vector, the Fig. 7 caption, stabilizer entropies, finite differences).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_liboracle.so")
_lock = threading.Lock()
_lib = None

ERR = {0: "ok", -1: "bad argument", -2: "out of memory", -6: "bad state"}


def build(force: bool = False) -> str:
    """Compile oracle.c into _liboracle.so (gcc, -O2, no arch-specific flags)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = C.CDLL(_LIB)
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C")
            i64p = np.ctypeslib.ndpointer(np.int64, flags="C")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C")
            u8p = np.ctypeslib.ndpointer(np.uint8, flags="C")
            vp = C.c_void_p
            sig = {
                "orc_gate_matrix": (C.c_int, [C.c_int, C.c_double, f64p]),
                "orc_asap": (C.c_int, [C.c_int, C.c_int, i32p, i32p]),
                "orc_partition": (C.c_int, [C.c_int, C.c_int, i32p, i32p, C.c_int, C.c_int, i64p,
                                            C.c_int, C.c_int, C.c_int, i32p, i32p, C.c_int,
                                            C.POINTER(C.c_int), C.POINTER(C.c_int)]),
                "orc_statevector": (C.c_int, [C.c_int, C.c_int, i32p, f64p, f64p]),
                "orc_cluster_unitary": (C.c_int, [C.c_int, C.c_int, C.c_int, i32p, f64p, i32p,
                                                  C.c_int, C.c_int, f64p]),
                "orc_svd": (C.c_int, [C.c_int, C.c_int, f64p, f64p, f64p]),
                "orc_mps_new": (vp, [C.c_int]),
                "orc_mps_free": (None, [vp]),
                "orc_mps_set_site": (C.c_int, [vp, C.c_int, C.c_longlong, C.c_longlong, f64p]),
                "orc_mps_set_lambda": (C.c_int, [vp, C.c_int, C.c_longlong, f64p]),
                "orc_mps_get_chi": (None, [vp, i64p]),
                "orc_mps_get_site": (None, [vp, C.c_int, f64p]),
                "orc_mps_get_lambda": (None, [vp, C.c_int, f64p]),
                "orc_mps_logF": (C.c_double, [vp]),
                "orc_mps_nlog": (C.c_int, [vp]),
                "orc_mps_get_log": (None, [vp, f64p]),
                "orc_mps_nstep": (C.c_int, [vp]),
                "orc_apply_1q": (C.c_int, [vp, C.c_int, f64p]),
                "orc_cluster_update": (C.c_int, [vp, C.c_int, C.c_int, f64p, C.c_int, C.c_double,
                                                 C.c_double, f64p, i32p]),
                "orc_run": (C.c_int, [vp, C.c_int, i32p, f64p, C.c_int, C.c_double, C.c_int,
                                      C.c_int, C.c_int, C.c_double]),
                "orc_amplitude": (C.c_int, [vp, u8p, f64p]),
                "orc_to_statevector": (C.c_int, [vp, f64p]),
                "orc_overlap": (C.c_int, [vp, vp, f64p]),
                "orc_stab_entropy": (C.c_int, [C.c_int, C.c_int, i32p, i32p]),
                "orc_mlp_forward": (C.c_int, [C.c_int] * 5 + [f64p, f64p, f64p]),
                "orc_mlp_loss_grad": (C.c_int, [C.c_int] * 5 + [f64p, f64p, i32p,
                                                               C.POINTER(C.c_double), f64p]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(rc):
    if rc is not None and rc < 0:
        raise RuntimeError(f"oracle error {rc}: {ERR.get(rc, '?')}")
    return rc


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128)).view(np.float64)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


# ---- App. A -----------------------------------------------------------------
def gate_matrix(kind: int, param: float = 0.0) -> np.ndarray:
    out = np.zeros(32, dtype=np.float64)
    d = _check(_L().orc_gate_matrix(int(kind), float(param), out))
    return out[: 2 * d * d].view(np.complex128).reshape(d, d)


# ---- Sec. II.A --------------------------------------------------------------
def asap_layers(n_qubits: int, gates: np.ndarray) -> tuple[np.ndarray, int]:
    g = _i32(gates).reshape(-1, 5)
    layer = np.zeros(max(len(g), 1), dtype=np.int32)
    nl = _check(_L().orc_asap(n_qubits, len(g), g.reshape(-1) if len(g) else np.zeros(5, np.int32), layer))
    return layer[: len(g)], nl


def statevector(circ) -> np.ndarray:
    out = np.zeros(2 << circ.n_qubits, dtype=np.float64)
    _check(_L().orc_statevector(circ.n_qubits, circ.n_gates, _i32(circ.gates).reshape(-1),
                                np.ascontiguousarray(circ.params, dtype=np.float64), out))
    return out.view(np.complex128)


# ---- Sec. III.A, Eqs. 6-8 ---------------------------------------------------
def partition(n_qubits, gates, layer, n_layers, start, chi, q_max, l_max, k_max):
    """Clusters [(q0, k), ...] and stop layer L* for one cluster-TEBD iteration."""
    g = _i32(gates).reshape(-1)
    cq = np.zeros(n_qubits, dtype=np.int32)
    ck = np.zeros(n_qubits, dtype=np.int32)
    nc, stop = C.c_int(0), C.c_int(0)
    _check(_L().orc_partition(n_qubits, len(layer), g, _i32(layer), int(n_layers), int(start),
                              np.ascontiguousarray(chi, dtype=np.int64), int(q_max), int(l_max),
                              int(k_max), cq, ck, n_qubits, C.byref(nc), C.byref(stop)))
    return [(int(cq[i]), int(ck[i])) for i in range(nc.value)], stop.value


def cluster_unitary(q0, k, circ, layer, lo, hi) -> np.ndarray:
    D = 1 << k
    out = np.zeros(2 * D * D, dtype=np.float64)
    _check(_L().orc_cluster_unitary(q0, k, circ.n_gates, _i32(circ.gates).reshape(-1),
                                    np.ascontiguousarray(circ.params, dtype=np.float64),
                                    _i32(layer), int(lo), int(hi), out))
    return out.view(np.complex128).reshape(D, D)


# ---- Fig. 3 building block --------------------------------------------------
def svd_right(M: np.ndarray):
    """Jacobi SVD: (s descending, Y with right singular vectors as columns)."""
    m, n = M.shape
    p = min(m, n)
    s = np.zeros(p)
    Y = np.zeros(2 * n * p)
    _check(_L().orc_svd(m, n, _c128(M).reshape(-1), s, Y))
    return s, Y.view(np.complex128).reshape(n, p)


def truncation_rank(s: np.ndarray, chi_max: int, cutoff: float, floor: float) -> int:
    """Rank kept by one truncated split (Sec. II.C, Eqs. 4-5): the smallest r
    whose discarded weight sum_{i>=r} s_i^2 stays within cutoff * sum s_i^2,
    then no more than the values above floor * s_0, at most chi_max, at least 1."""
    s2 = np.asarray(s, dtype=np.float64) ** 2
    W = s2.sum()
    r = len(s2)
    if cutoff > 0:
        tail = np.cumsum(s2[::-1])[::-1]          # tail[i] = sum_{j>=i} s_j^2
        over = np.nonzero(tail[1:] > cutoff * W)[0]
        r = int(over[-1]) + 2 if len(over) else 1
    r = min(r, int(np.sum(s > floor * s[0])), chi_max)
    return max(r, 1)


def split_fidelity(M: np.ndarray, w: np.ndarray, chi_max: int, cutoff: float, floor: float = 1e-13):
    """One truncated split of the Schmidt-weighted matrix diag(w) M (Sec. II.C):
    returns (r, f, W, s) with s the singular values of diag(w) M, W = sum s^2,
    r the kept rank and f = sum_{i<r} s_i^2 / W the split's fidelity (Eq. 4).
    The SVD is LAPACK's (numpy), a library step; sizes up to a few thousand."""
    A = np.asarray(w, dtype=np.float64)[:, None] * np.asarray(M, dtype=np.complex128)
    s = np.linalg.svd(A, compute_uv=False)
    r = truncation_rank(s, chi_max, cutoff, floor)
    W = float(np.sum(s * s))
    f = float(np.sum(s[:r] ** 2) / W) if W > 0 else 1.0
    return r, f, W, s


def split_chain(theta: np.ndarray, lam_l: np.ndarray, chi_max: int, cutoff: float,
                floor: float = 1e-13):
    """The k-1 truncated splits of one cluster update (Sec. III.A, Fig. 2 and
    Fig. 3), right to left, in the gauge of MPS.cluster_update: split j
    factors diag(lambda_L) Rbar_j (chi_L 2^j x 2 r_{j+1}); the kept right
    singular vectors give the new site, the unweighted remainder Rbar_j Y_r /
    sqrt(kept) feeds split j-1.  theta: (chi_L, 2^k, chi_R) with the cluster
    unitary applied and without the left weights.  The SVD is LAPACK's (numpy),
    a library step; sizes up to a few thousand.  Returns one dict per split,
    rightmost bond first: j (bond q0 + j), m, n, r, f (Eq. 4), W, s, lam."""
    th = np.asarray(theta, dtype=np.complex128)
    cl, D, cr = th.shape
    k = int(round(np.log2(D)))
    lam_l = np.asarray(lam_l, dtype=np.float64)
    R, rdim, out = th.reshape(-1), cr, []
    for j in range(k - 1, 0, -1):
        m, n = cl << j, 2 * rdim
        Mb = R.reshape(m, n)
        w = np.repeat(lam_l, 1 << j)
        _, s, Vh = np.linalg.svd(w[:, None] * Mb, full_matrices=False)
        r = truncation_rank(s, chi_max, cutoff, floor)
        W = float(np.sum(s * s))
        kept = float(np.sum(s[:r] ** 2))
        out.append({"j": j, "m": m, "n": n, "r": r, "f": kept / W if W > 0 else 1.0, "W": W,
                    "s": s, "lam": s[:r] / np.sqrt(kept)})
        R = (Mb @ Vh[:r].conj().T / np.sqrt(kept)).reshape(-1)
        rdim = r
    return out


def _positive_floor(floor: float):
    """The numerical-zero floor of the truncation rule must be positive:
    with none, singular values at the rounding level are kept, and their
    singular vectors are not determined."""
    if not floor > 0:
        raise ValueError("floor must be positive (singular values <= floor * s_1 are numerical zeros)")


# ---- MPS (Vidal form, Sec. II.B-II.C, III.A) --------------------------------
class MPS:
    """Oracle MPS: right-canonical sites B_q (chi_q, 2, chi_{q+1}) + spectra."""

    def __init__(self, n_qubits: int):
        self.n = n_qubits
        self._h = _L().orc_mps_new(n_qubits)
        if not self._h:
            raise MemoryError

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_mps_free(h)
            self._h = None

    @classmethod
    def from_arrays(cls, sites, lams):
        m = cls(len(sites))
        for q, s in enumerate(sites):
            s = np.asarray(s, dtype=np.complex128)
            _check(_L().orc_mps_set_site(m._h, q, s.shape[0], s.shape[2], _c128(s).reshape(-1)))
        for b, l in enumerate(lams):
            l = np.ascontiguousarray(l, dtype=np.float64)
            _check(_L().orc_mps_set_lambda(m._h, b, len(l), l))
        return m

    def chi(self) -> np.ndarray:
        out = np.zeros(self.n + 1, dtype=np.int64)
        _L().orc_mps_get_chi(self._h, out)
        return out

    def site(self, q: int) -> np.ndarray:
        c = self.chi()
        out = np.zeros(2 * c[q] * 2 * c[q + 1])
        _L().orc_mps_get_site(self._h, q, out)
        return out.view(np.complex128).reshape(c[q], 2, c[q + 1])

    def lam(self, b: int) -> np.ndarray:
        out = np.zeros(self.chi()[b])
        _L().orc_mps_get_lambda(self._h, b, out)
        return out

    @property
    def logF(self) -> float:
        return _L().orc_mps_logF(self._h)

    @property
    def n_steps(self) -> int:
        return _L().orc_mps_nstep(self._h)

    def split_log(self) -> np.ndarray:
        """Rows (step, q0, k, bond, m, n, r, f_j, W) for every split performed."""
        nl = _L().orc_mps_nlog(self._h)
        out = np.zeros(9 * max(nl, 1))
        _L().orc_mps_get_log(self._h, out)
        return out[: 9 * nl].reshape(nl, 9)

    def apply_1q(self, q: int, u: np.ndarray):
        _check(_L().orc_apply_1q(self._h, q, _c128(u).reshape(-1)))

    def cluster_update(self, q0, k, U, chi_max, cutoff, floor=1e-13):
        _positive_floor(floor)
        f = np.zeros(max(k - 1, 1))
        r = np.zeros(max(k - 1, 1), dtype=np.int32)
        _check(_L().orc_cluster_update(self._h, q0, k, _c128(U).reshape(-1), int(chi_max),
                                       float(cutoff), float(floor), f, r))
        return f[: k - 1], r[: k - 1]

    def run(self, circ, chi_max, cutoff, q_max, l_max=0, k_max=0, floor=1e-13):
        _positive_floor(floor)
        _check(_L().orc_run(self._h, circ.n_gates, _i32(circ.gates).reshape(-1),
                            np.ascontiguousarray(circ.params, dtype=np.float64), int(chi_max),
                            float(cutoff), int(q_max), int(l_max), int(k_max), float(floor)))
        return self

    def amplitude(self, bits) -> complex:
        out = np.zeros(2)
        _check(_L().orc_amplitude(self._h, np.ascontiguousarray(bits, dtype=np.uint8), out))
        return complex(out[0], out[1])

    def statevector(self) -> np.ndarray:
        out = np.zeros(2 << self.n)
        _check(_L().orc_to_statevector(self._h, out))
        return out.view(np.complex128)

    def overlap(self, other: "MPS") -> complex:
        out = np.zeros(2)
        _check(_L().orc_overlap(self._h, other._h, out))
        return complex(out[0], out[1])


def simulate(circ, chi_max, cutoff, q_max, l_max=0, k_max=0, floor=1e-13) -> MPS:
    """Cluster-TEBD from |0...0> over the whole circuit (Sec. III.A)."""
    return MPS(circ.n_qubits).run(circ, chi_max, cutoff, q_max, l_max, k_max, floor)


# ---- Sec. III.B: virtual MPS (Eq. 9) and adaptive grouping (Eqs. 10-11) -----
def virtual_bonds(n: int, gates: np.ndarray, layer: np.ndarray, layer_start: int, l_max: int,
                  chi, chi_max: int):
    """Eq. 9: for every bond b = 0..n (b qubits on its left), E(b) = number of
    multi-qubit gates with layer_start < layer <= layer_start + l_max (all later
    layers for l_max <= 0) that span bond b, and the virtual bond dimension
    min(2^E(b) chi_b, chi_max, 2^min(b, n - b)).  Plain loops."""
    E = [0] * (n + 1)
    for g, L in zip(np.asarray(gates).reshape(-1, 5), layer):
        nq = int(g[0])
        if nq < 2 or L <= layer_start or (l_max > 0 and L > layer_start + l_max):
            continue
        qs = [int(q) for q in g[1:1 + nq]]
        for b in range(min(qs) + 1, max(qs) + 1):
            E[b] += 1
    out = []
    for b in range(n + 1):
        out.append(min(2 ** E[b] * int(chi[b]), chi_max, 2 ** min(b, n - b)))
    return np.array(out, dtype=np.int64), np.array(E, dtype=np.int64)


def grouping(chi_v, q_max: int, imbalance: float = 1.0 / 3.0):
    """Eqs. 10-11: recursive bipartitioning of the virtual MPS.  A segment of
    sites [lo, hi) is accepted when its qubit count plus log2 of its two
    boundary bonds (1 at the chain ends) is at most q_max; otherwise it is cut
    at its bond of smallest virtual dimension, among cuts leaving each part at
    most (1 + imbalance) * ceil(size / 2) sites (ties: the most central, then
    the leftmost), and both parts are examined in turn.  Returns the group
    start sites in ascending order; raises ValueError when a single site does
    not fit."""
    chi_v = [int(x) for x in chi_v]
    n = len(chi_v) - 1

    def bond(b):
        return 1 if b in (0, n) else chi_v[b]

    def fits(lo, hi):
        # (hi - lo) + log2 chi_lo + log2 chi_hi <= q_max, in integers
        return (1 << (hi - lo)) * bond(lo) * bond(hi) <= (1 << q_max) if q_max >= 0 else False

    def split(lo, hi):
        if fits(lo, hi):
            return [lo]
        size = hi - lo
        if size == 1:
            raise ValueError(f"site {lo} does not fit")
        limit = math.floor((1.0 + imbalance) * ((size + 1) // 2) + 1e-9)
        cands = [k for k in range(lo + 1, hi) if k - lo <= limit and hi - k <= limit]
        k = min(cands, key=lambda c: (bond(c), abs(2 * c - (lo + hi)), c))
        return split(lo, k) + split(k, hi)

    return split(0, n)


# ---- Gottesman-Knill pin ----------------------------------------------------
def stabilizer_entropies(circ) -> np.ndarray:
    """S_b (bits) for b = 0..n of a Clifford circuit's output state."""
    out = np.zeros(circ.n_qubits + 1, dtype=np.int32)
    _check(_L().orc_stab_entropy(circ.n_qubits, circ.n_gates, _i32(circ.gates).reshape(-1), out))
    return out


# ---- rank-predictor network reference ---------------------------------------
def mlp_sizes(F, H1, H2, NB):
    return [(H1, F), (H1,), (H2, H1), (H2,), (NB, H2), (NB,)]


def mlp_nparams(F, H1, H2, NB):
    return H1 * F + H1 + H2 * H1 + H2 + NB * H2 + NB


def mlp_forward(P, X, F, H1, H2, NB):
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.zeros(X.shape[0] * NB)
    _check(_L().orc_mlp_forward(X.shape[0], F, H1, H2, NB, np.ascontiguousarray(P, dtype=np.float64),
                                X.reshape(-1), out))
    return out.reshape(-1, NB)


def mlp_loss_grad(P, X, y, F, H1, H2, NB):
    X = np.ascontiguousarray(X, dtype=np.float64)
    g = np.zeros(mlp_nparams(F, H1, H2, NB))
    loss = C.c_double(0)
    _check(_L().orc_mlp_loss_grad(X.shape[0], F, H1, H2, NB, np.ascontiguousarray(P, dtype=np.float64),
                                  X.reshape(-1), _i32(y), C.byref(loss), g))
    return loss.value, g
