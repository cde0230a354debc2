"""GB300 cluster-TEBD cluster update (arXiv 2502.19289, Sec. III.A).

Thin ctypes binding of ``libctebd.so`` (C ABI in ``include/ctebd.h``).  This
module only marshals arguments: partition, cluster unitaries, contraction,
truncated splits and observables all run inside the library (host C++ for the
partition and unitaries, CUDA kernels for everything on the state).  There is
no CPU fallback: importing this package without the built library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libctebd.so")

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NUMERIC, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
FP64, FP32 = 0, 1


class CtebdError(RuntimeError):
    pass


class Config(C.Structure):
    _fields_ = [("n_qubits", C.c_int), ("chi_max", C.c_int), ("cutoff", C.c_double),
                ("q_max", C.c_int), ("l_max", C.c_int), ("k_max", C.c_int),
                ("precision", C.c_int), ("sketch_oversample", C.c_int),
                ("power_iters", C.c_int), ("use_rank_model", C.c_int), ("seed", C.c_uint64)]


class Gate(C.Structure):
    _fields_ = [("layer", C.c_int), ("n_q", C.c_int), ("q", C.c_int * 3), ("kind", C.c_int),
                ("param", C.c_double)]


class Cluster(C.Structure):
    _fields_ = [("q0", C.c_int), ("k", C.c_int), ("layer_lo", C.c_int), ("layer_hi", C.c_int),
                ("rank_hint", C.c_int * 11)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python paper_2502_19289_gb300/build.py` "
            "(nvcc, sm_103a). There is no CPU fallback.")
    lib = C.CDLL(LIB_PATH)
    P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    sig = {
        "mps_create": [C.POINTER(Config), P, C.POINTER(P)],
        "mps_destroy": [P],
        "assign_layers": [C.POINTER(Gate), I, I, C.POINTER(I)],
        "cluster_partition": [C.POINTER(Gate), I, I, C.POINTER(I), C.POINTER(Config),
                              C.POINTER(Cluster), I, C.POINTER(I), C.POINTER(I)],
        "cluster_unitary": [C.POINTER(Gate), I, C.POINTER(Cluster), C.POINTER(D)],
        "apply_1q": [P, I, C.POINTER(D)],
        "apply_singletons": [P, C.POINTER(Gate), I, C.POINTER(Cluster), I, I, I],
        "apply_cluster": [P, C.POINTER(Cluster), C.POINTER(D)],
        "truncate_split": [P, C.POINTER(Cluster), C.POINTER(D)],
        "step": [P, C.POINTER(Cluster), I, C.POINTER(C.POINTER(D)), C.POINTER(D)],
        "fidelity": [P, C.POINTER(D)],
        "amplitude": [P, C.POINTER(C.c_uint8), C.POINTER(D), C.POINTER(D)],
        "mps_bond_dims": [P, C.POINTER(I)],
        "mps_to_host": [P, I, C.POINTER(D), S],
        "mps_lambda_to_host": [P, I, C.POINTER(D), S],
        "mps_load": [P, C.POINTER(I), C.POINTER(C.POINTER(D)), C.POINTER(C.POINTER(D))],
        "mps_load_device": [P, C.POINTER(I), C.POINTER(P), C.POINTER(P)],
        "mps_split_log": [P, C.POINTER(D), I, C.POINTER(I)],
        "mps_sketch_stats": [P, C.POINTER(D)],
        "mps_solver_stats": [P, C.POINTER(D)],
        "cluster_rank_bounds": [C.POINTER(Gate), I, C.POINTER(Cluster), C.POINTER(I), C.POINTER(I)],
        "ctebd_last_error": [C.c_char_p, S],
        "ctebd_profile": [P, I],
        "ctebd_profile_read": [P, C.POINTER(D), I, C.POINTER(I)],
        "ctebd_kernel_name": [I, C.c_char_p, S],
        "split2_noalloc": [P, P, I, I, I, D, P, P, P, C.POINTER(I), C.POINTER(D), P],
        "rank_features": [C.POINTER(Gate), I, C.POINTER(Cluster), C.POINTER(I), C.POINTER(D),
                          C.POINTER(Config), C.POINTER(C.c_float)],
        "mps_bond_entropies": [P, C.POINTER(D)],
        "rank_model_load": [P, C.POINTER(C.c_float), S],
        "rank_model_predict": [P, C.POINTER(C.c_float), I, C.POINTER(I), C.POINTER(I)],
        "mlp_nparams_abi": [],
        "tc_cgemm": [P, P, P, I, I, I, P],
        "ctebd_set_tensor_cores": [I],
        "ctebd_set_sweep_graphs": [I],
        "ctebd_set_max_sweeps": [I],
        "ctebd_max_sweeps": [],
        "virtual_mps_bonds": [C.POINTER(Gate), I, I, I, I, C.POINTER(I), I, C.POINTER(I), C.POINTER(I)],
        "adaptive_grouping": [C.POINTER(I), I, I, D, C.POINTER(I), I, C.POINTER(I)],
        "ctebd_measure_fma": [I, C.POINTER(D), C.POINTER(D), C.POINTER(I)],
        "mlp_forward": [P, P, I, P, P],
        "mlp_loss_grad": [P, P, P, I, P, P, P],
        "mlp_adam": [P, P, P, P, I, C.c_float, I, P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    return lib


_lib = _load()
lib = _lib


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    _lib.ctebd_last_error(buf, 1024)
    return buf.value.decode(errors="replace")


def _check(rc: int, what: str):
    if rc != OK:
        raise CtebdError(f"{what} failed ({rc}): {last_error()}")


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def make_config(n_qubits, chi_max, cutoff, q_max, l_max=0, k_max=0, precision=FP32,
                sketch_oversample=0, power_iters=1, use_rank_model=0, seed=1234) -> Config:
    return Config(n_qubits, chi_max, cutoff, q_max, l_max, k_max, precision,
                  sketch_oversample, power_iters, use_rank_model, seed)


def gates_from_arrays(gates5: np.ndarray, params: np.ndarray):
    """Input-format gate rows (n_q, q0, q1, q2, kind) -> ctebd_gate array."""
    g = np.asarray(gates5, dtype=np.int32).reshape(-1, 5)
    arr = (Gate * max(len(g), 1))()
    for i, (nq, a, b, c, kind) in enumerate(g):
        arr[i].layer = 0
        arr[i].n_q = int(nq)
        arr[i].q[0], arr[i].q[1], arr[i].q[2] = int(a), int(b), int(c)
        arr[i].kind = int(kind)
        arr[i].param = float(params[i])
    return arr, len(g)


def assign_layers(gates, n_gates, n_qubits) -> int:
    nl = C.c_int(0)
    _check(_lib.assign_layers(gates, n_gates, n_qubits, C.byref(nl)), "assign_layers")
    return nl.value


def cluster_partition(gates, n_gates, layer_start, chi, cfg: Config):
    chi = np.ascontiguousarray(chi, dtype=np.int32)
    cap = max(cfg.n_qubits, 1)
    out = (Cluster * cap)()
    n_out, stop = C.c_int(0), C.c_int(0)
    _check(_lib.cluster_partition(gates, n_gates, layer_start, _ip(chi), C.byref(cfg), out, cap,
                                  C.byref(n_out), C.byref(stop)), "cluster_partition")
    return [out[i] for i in range(n_out.value)], stop.value


def cluster_rank_bounds(gates, n_gates, cl: Cluster, chi) -> np.ndarray:
    """Eq. 9 rank bound per internal bond of the cluster (left to right)."""
    chi = np.ascontiguousarray(chi, dtype=np.int32)
    out = np.zeros(max(cl.k - 1, 1), dtype=np.int32)
    _check(_lib.cluster_rank_bounds(gates, n_gates, C.byref(cl), _ip(chi), _ip(out)),
           "cluster_rank_bounds")
    return out[: cl.k - 1]


def virtual_mps_bonds(gates, n_gates, n_qubits, layer_start, l_max, chi, chi_max):
    """Eq. 9 virtual-MPS bond dimensions (N+1) and the entangling-gate counts E(b)."""
    chi = np.ascontiguousarray(chi, dtype=np.int32)
    out = np.zeros(n_qubits + 1, dtype=np.int32)
    ent = np.zeros(n_qubits + 1, dtype=np.int32)
    _check(_lib.virtual_mps_bonds(gates, n_gates, n_qubits, int(layer_start), int(l_max), _ip(chi),
                                  int(chi_max), _ip(out), _ip(ent)), "virtual_mps_bonds")
    return out, ent


def adaptive_grouping(chi_v, q_max, imbalance=1.0 / 3.0):
    """Eqs. 10-11 recursive min-cut grouping: the first site of every group."""
    chi_v = np.ascontiguousarray(chi_v, dtype=np.int32)
    n = len(chi_v) - 1
    out = np.zeros(max(n, 1), dtype=np.int32)
    ng = C.c_int(0)
    _check(_lib.adaptive_grouping(_ip(chi_v), n, int(q_max), float(imbalance), _ip(out), len(out),
                                  C.byref(ng)), "adaptive_grouping")
    return out[: ng.value]


def rank_features(gates, n_gates, cl: Cluster, chi, entropy, cfg: Config) -> np.ndarray:
    """16 features per split of the cluster (rows: bonds q0+1 .. q0+k-1)."""
    chi = np.ascontiguousarray(chi, dtype=np.int32)
    ent = np.ascontiguousarray(entropy, dtype=np.float64)
    out = np.zeros((max(cl.k - 1, 1), 16), dtype=np.float32)
    _check(_lib.rank_features(gates, n_gates, C.byref(cl), _ip(chi), _dp(ent), C.byref(cfg),
                              out.ctypes.data_as(C.POINTER(C.c_float))), "rank_features")
    return out[: cl.k - 1]


def set_tensor_cores(mode: int):
    """FP32 GEMM policy: 0 CUDA cores only, 1 batches above 2 GFLOP (problems under 64 rows
    on the CUDA cores; default), 2 always."""
    _check(_lib.ctebd_set_tensor_cores(int(mode)), "ctebd_set_tensor_cores")


def set_sweep_graphs(mode: int):
    """Where an eigen-solve's sweep loop runs: 1 (default) on the device as one
    CUDA graph for batches at least 16 Jacobi blocks wide, from the host for
    narrower ones; 2 on the device for every batch; 0 from the host for every
    batch.  Process-wide (ctebd_set_sweep_graphs)."""
    _check(_lib.ctebd_set_sweep_graphs(int(mode)), "ctebd_set_sweep_graphs")


def set_max_sweeps(n: int):
    """Sweep cap of the Jacobi eigen-solves (default 60); a solve still rotating at
    the cap makes the split fail with CTEBD_ERR_NUMERIC; process-wide."""
    _check(_lib.ctebd_set_max_sweeps(int(n)), "ctebd_set_max_sweeps")


def max_sweeps() -> int:
    """The current sweep cap of the Jacobi eigen-solves."""
    return int(_lib.ctebd_max_sweeps())


def measure_fma(repeats: int = 5):
    """Measured FP32 CUDA-core throughput: (best TFLOP/s, mean TFLOP/s, SM count)."""
    best, mean, sms = C.c_double(0), C.c_double(0), C.c_int(0)
    _check(_lib.ctebd_measure_fma(int(repeats), C.byref(best), C.byref(mean), C.byref(sms)),
           "ctebd_measure_fma")
    return best.value, mean.value, sms.value


def tc_cgemm(A_ptr, B_ptr, C_ptr, M, K, N, stream=None):
    """Complex64 product on the tensor cores (validation of the tile engine)."""
    _check(_lib.tc_cgemm(C.c_void_p(A_ptr), C.c_void_p(B_ptr), C.c_void_p(C_ptr), M, K, N,
                         C.c_void_p(stream or 0)), "tc_cgemm")


def mlp_nparams() -> int:
    return _lib.mlp_nparams_abi()


def mlp_forward(params_ptr, X_ptr, B, logits_ptr, stream=None):
    _check(_lib.mlp_forward(C.c_void_p(params_ptr), C.c_void_p(X_ptr), B, C.c_void_p(logits_ptr),
                            C.c_void_p(stream or 0)), "mlp_forward")


def mlp_loss_grad(params_ptr, X_ptr, y_ptr, B, grad_ptr, loss_ptr, stream=None):
    _check(_lib.mlp_loss_grad(C.c_void_p(params_ptr), C.c_void_p(X_ptr), C.c_void_p(y_ptr), B,
                              C.c_void_p(grad_ptr), C.c_void_p(loss_ptr), C.c_void_p(stream or 0)),
           "mlp_loss_grad")


def mlp_adam(params_ptr, grad_ptr, m1_ptr, m2_ptr, n, lr, t, stream=None):
    _check(_lib.mlp_adam(C.c_void_p(params_ptr), C.c_void_p(grad_ptr), C.c_void_p(m1_ptr),
                         C.c_void_p(m2_ptr), n, C.c_float(lr), t, C.c_void_p(stream or 0)), "mlp_adam")


def cluster_unitary(gates, n_gates, cl: Cluster) -> np.ndarray:
    D = 1 << cl.k
    U = np.zeros(2 * D * D)
    _check(_lib.cluster_unitary(gates, n_gates, C.byref(cl), _dp(U)), "cluster_unitary")
    return U.view(np.complex128).reshape(D, D)


class MPS:
    """Device MPS handle (right-canonical sites + bond spectra)."""

    def __init__(self, cfg: Config, stream=None):
        self.cfg = cfg
        self.n = cfg.n_qubits
        h = C.c_void_p()
        _check(_lib.mps_create(C.byref(cfg), C.c_void_p(stream or 0), C.byref(h)), "mps_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            _lib.mps_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- state access ---------------------------------------------------
    def bond_dims(self) -> np.ndarray:
        chi = np.zeros(self.n + 1, dtype=np.int32)
        _check(_lib.mps_bond_dims(self._h, _ip(chi)), "mps_bond_dims")
        return chi

    def site(self, q: int) -> np.ndarray:
        chi = self.bond_dims()
        buf = np.zeros(2 * chi[q] * 2 * chi[q + 1])
        _check(_lib.mps_to_host(self._h, q, _dp(buf), buf.size), "mps_to_host")
        return buf.view(np.complex128).reshape(chi[q], 2, chi[q + 1])

    def lam(self, b: int) -> np.ndarray:
        chi = self.bond_dims()
        buf = np.zeros(max(chi[b], 1))
        _check(_lib.mps_lambda_to_host(self._h, b, _dp(buf), buf.size), "mps_lambda_to_host")
        return buf[: chi[b]]

    def load(self, chi, sites, lams):
        chi = np.ascontiguousarray(chi, dtype=np.int32)
        s = [np.ascontiguousarray(x, dtype=np.complex128).view(np.float64).reshape(-1) for x in sites]
        l = [np.ascontiguousarray(x, dtype=np.float64) for x in lams]
        sp = (C.POINTER(C.c_double) * len(s))(*[_dp(x) for x in s])
        lp = (C.POINTER(C.c_double) * len(l))(*[_dp(x) for x in l])
        _check(_lib.mps_load(self._h, _ip(chi), sp, lp), "mps_load")

    def load_device(self, chi, site_ptrs, lam_ptrs):
        chi = np.ascontiguousarray(chi, dtype=np.int32)
        sp = (C.c_void_p * len(site_ptrs))(*site_ptrs)
        lp = (C.c_void_p * len(lam_ptrs))(*lam_ptrs)
        _check(_lib.mps_load_device(self._h, _ip(chi), sp, lp), "mps_load_device")

    def bond_entropies(self) -> np.ndarray:
        out = np.zeros(self.n + 1)
        _check(_lib.mps_bond_entropies(self._h, _dp(out)), "mps_bond_entropies")
        return out

    def load_rank_model(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(_lib.rank_model_load(self._h, p.ctypes.data_as(C.POINTER(C.c_float)), p.size),
               "rank_model_load")

    def predict_hints(self, features, bounds) -> np.ndarray:
        X = np.ascontiguousarray(features, dtype=np.float32).reshape(-1, 16)
        b = np.ascontiguousarray(bounds, dtype=np.int32)
        out = np.zeros(len(b), dtype=np.int32)
        _check(_lib.rank_model_predict(self._h, X.ctypes.data_as(C.POINTER(C.c_float)), len(b),
                                       _ip(b), _ip(out)), "rank_model_predict")
        return out

    def fidelity(self) -> float:
        F = C.c_double(0)
        _check(_lib.fidelity(self._h, C.byref(F)), "fidelity")
        return F.value

    def amplitude(self, bits) -> complex:
        b = np.ascontiguousarray(bits, dtype=np.uint8)
        re, im = C.c_double(0), C.c_double(0)
        _check(_lib.amplitude(self._h, b.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(re),
                              C.byref(im)), "amplitude")
        return complex(re.value, im.value)

    def split_log(self) -> np.ndarray:
        n = C.c_int(0)
        _check(_lib.mps_split_log(self._h, None, 0, C.byref(n)), "mps_split_log")
        rows = np.zeros(14 * max(n.value, 1))
        _check(_lib.mps_split_log(self._h, _dp(rows), n.value, C.byref(n)), "mps_split_log")
        return rows[: 14 * n.value].reshape(-1, 14)

    def sketch_stats(self):
        out = np.zeros(2)
        _check(_lib.mps_sketch_stats(self._h, _dp(out)), "mps_sketch_stats")
        return int(out[0]), int(out[1])

    def solver_stats(self):
        """(refinement passes accepted at the sweep cap, their largest
        last-sweep moved weight relative to the trace)."""
        out = np.zeros(2)
        _check(_lib.mps_solver_stats(self._h, _dp(out)), "mps_solver_stats")
        return int(out[0]), float(out[1])

    # --- the cluster update ----------------------------------------------
    def apply_1q(self, q: int, u: np.ndarray):
        u = np.ascontiguousarray(u, dtype=np.complex128).view(np.float64).reshape(-1)
        _check(_lib.apply_1q(self._h, q, _dp(u)), "apply_1q")

    def apply_singletons(self, gates, n_gates, clusters, lo, hi):
        arr = (Cluster * max(len(clusters), 1))(*clusters)
        _check(_lib.apply_singletons(self._h, gates, n_gates, arr, len(clusters), lo, hi),
               "apply_singletons")

    def apply_cluster(self, cl: Cluster, U: np.ndarray):
        U = np.ascontiguousarray(U, dtype=np.complex128).view(np.float64).reshape(-1)
        _check(_lib.apply_cluster(self._h, C.byref(cl), _dp(U)), "apply_cluster")

    def truncate_split(self, cl: Cluster) -> np.ndarray:
        f = np.zeros(max(cl.k - 1, 1))
        _check(_lib.truncate_split(self._h, C.byref(cl), _dp(f)), "truncate_split")
        return f[: cl.k - 1]

    def step(self, clusters, Us) -> np.ndarray:
        n = len(clusters)
        arr = (Cluster * max(n, 1))(*clusters)
        Uf = [np.ascontiguousarray(U, dtype=np.complex128).view(np.float64).reshape(-1) for U in Us]
        up = (C.POINTER(C.c_double) * max(n, 1))(*[_dp(u) for u in Uf])
        f = np.zeros(max(sum(c.k - 1 for c in clusters), 1))
        _check(_lib.step(self._h, arr, n, up, _dp(f)), "step")
        return f[: sum(c.k - 1 for c in clusters)]


def split2_noalloc(theta_ptr, lam_ptr, chi_l, chi_r, chi_max, cutoff, site_l_ptr, site_r_ptr,
                   lam_out_ptr, stream=None):
    """Two-site split without device allocation (device pointers in and out).

    Returns (r, f).  See include/ctebd.h for limits and scratch semantics."""
    r, f = C.c_int(0), C.c_double(0)
    _check(_lib.split2_noalloc(C.c_void_p(theta_ptr), C.c_void_p(lam_ptr), chi_l, chi_r, chi_max,
                               cutoff, C.c_void_p(site_l_ptr), C.c_void_p(site_r_ptr),
                               C.c_void_p(lam_out_ptr), C.byref(r), C.byref(f),
                               C.c_void_p(stream or 0)), "split2_noalloc")
    return r.value, f.value


# C-style aliases with the ABI's names
def mps_create(cfg: Config, stream=None) -> MPS:
    return MPS(cfg, stream)


def apply_cluster(mps: MPS, cl: Cluster, U):
    return mps.apply_cluster(cl, U)


def truncate_split(mps: MPS, cl: Cluster):
    return mps.truncate_split(cl)


def step(mps: MPS, clusters, Us):
    return mps.step(clusters, Us)


def fidelity(mps: MPS) -> float:
    return mps.fidelity()


def amplitude(mps: MPS, bits) -> complex:
    return mps.amplitude(bits)


def _by_layer(gates, n_gates):
    """A copy of a layered gate array in layer order (stable: the given order
    within a layer).  The partition, the cluster unitaries and the one-qubit
    pass find a layer range in such an array by binary search instead of
    sorting the whole list on every call; their results are the same."""
    out = (Gate * max(n_gates, 1))()
    if n_gates:
        layer = np.array([gates[i].layer for i in range(n_gates)], dtype=np.int64)
        order = np.argsort(layer, kind="stable")
        sz = C.sizeof(Gate)
        src = np.frombuffer((C.c_char * (sz * n_gates)).from_address(C.addressof(gates)), dtype=np.uint8)
        dst = np.frombuffer((C.c_char * (sz * n_gates)).from_address(C.addressof(out)), dtype=np.uint8)
        dst[:] = src.reshape(n_gates, sz)[order].reshape(-1)
    return out


class Circuit:
    """A circuit in the library's gate format, layered (Sec. II.A).  ``gates``
    keeps the given order; ``gates_by_layer`` holds the same gates in layer
    order, which the iteration drivers pass to the library."""

    def __init__(self, n_qubits: int, gates5, params):
        self.n = n_qubits
        self.gates, self.n_gates = gates_from_arrays(gates5, params)
        self.n_layers = assign_layers(self.gates, self.n_gates, n_qubits)
        self.gates_by_layer = _by_layer(self.gates, self.n_gates)


def run_iteration(mps: MPS, circ: Circuit, start: int, hint_fn=None):
    """One cluster-TEBD iteration (Sec. III.A) from layer ``start``.

    With sketching enabled (FP32, sketch_oversample > 0) each cluster gets
    rank hints: ``hint_fn(clusters, chi)`` if given (the learned predictor,
    see ``rank_model.make_hint_fn``), else the Eq. 9 bound.  Returns (clusters, stop layer, per-split f)."""
    chi = mps.bond_dims()
    g = circ.gates_by_layer
    clusters, stop = cluster_partition(g, circ.n_gates, start, chi, mps.cfg)
    if mps.cfg.sketch_oversample > 0 and mps.cfg.precision == FP32 and clusters:
        hints = (hint_fn(clusters, chi) if hint_fn else
                 [cluster_rank_bounds(g, circ.n_gates, c, chi) for c in clusters])
        for c, hint in zip(clusters, hints):
            for j, h in enumerate(hint[:11]):
                c.rank_hint[j] = int(h)
    mps.apply_singletons(g, circ.n_gates, clusters, start, stop)
    Us = [cluster_unitary(g, circ.n_gates, c) for c in clusters]
    f = mps.step(clusters, Us) if clusters else np.zeros(0)
    return clusters, stop, f


def simulate(circ: Circuit, cfg: Config, stream=None, callback=None, hint_fn=None) -> MPS:
    """Cluster-TEBD from |0...0> over the whole circuit (Sec. III.A loop)."""
    mps = MPS(cfg, stream)
    start = 0
    while start < circ.n_layers:
        clusters, stop, f = run_iteration(mps, circ, start, hint_fn)
        if callback:
            callback(start, stop, clusters, f)
        start = stop
    return mps


class PackedCircuits:
    """Independent circuits laid side by side on one MPS (cfg5-style packing).

    Circuit i occupies qubits [offset_i, offset_i + n_i); no gate crosses the
    boundaries, so the bonds between circuits stay at dimension 1.  Every
    circuit keeps its own partition and stop layer (Sec. III.A applied per
    circuit); one iteration advances every unfinished circuit by one of its
    own iterations, and the clusters of all circuits go into the same batched
    launches."""

    def __init__(self, circuits):
        self.locals = []
        self.offsets = []
        off = 0
        rows, params = [], []
        for n, gates5, prm in circuits:
            g = np.asarray(gates5, dtype=np.int32).reshape(-1, 5).copy()
            self.locals.append(Circuit(n, g, prm))
            self.offsets.append(off)
            gs = g.copy()
            for col in (1, 2, 3):
                gs[:, col] = np.where(gs[:, col] >= 0, gs[:, col] + off, -1)
            rows.append(gs)
            params.append(np.asarray(prm, dtype=np.float64))
            off += n
        self.n = off
        self.globals = [Circuit(self.n, r, p) for r, p in zip(rows, params)]
        self.start = [0] * len(circuits)

    def done(self) -> bool:
        return all(s >= c.n_layers for s, c in zip(self.start, self.locals))

    def iteration(self, mps: "MPS", cfg_local):
        """One iteration of every unfinished circuit; returns clusters stepped."""
        chi = mps.bond_dims()
        all_clusters, Us = [], []
        for i, (loc, glob, off) in enumerate(zip(self.locals, self.globals, self.offsets)):
            if self.start[i] >= loc.n_layers:
                continue
            cfg_local.n_qubits = loc.n
            cl, stop = cluster_partition(loc.gates_by_layer, loc.n_gates, self.start[i],
                                         chi[off:off + loc.n + 1], cfg_local)
            for c in cl:
                c.q0 += off
            gg = glob.gates_by_layer
            mps.apply_singletons(gg, glob.n_gates, cl, self.start[i], stop)
            if mps.cfg.sketch_oversample > 0 and mps.cfg.precision == FP32:
                for c in cl:
                    for j, h in enumerate(cluster_rank_bounds(gg, glob.n_gates, c, chi)[:11]):
                        c.rank_hint[j] = int(h)
            Us.extend(cluster_unitary(gg, glob.n_gates, c) for c in cl)
            all_clusters.extend(cl)
            self.start[i] = stop
        if all_clusters:
            mps.step(all_clusters, Us)
        return all_clusters


def simulate_packed(circuits, cfg: Config, stream=None, callback=None):
    """Run several independent circuits packed on one MPS; returns (mps, packing)."""
    pk = PackedCircuits(circuits)
    big = Config.from_buffer_copy(cfg)
    big.n_qubits = pk.n
    mps = MPS(big, stream)
    local = Config.from_buffer_copy(cfg)
    while not pk.done():
        cl = pk.iteration(mps, local)
        if callback:
            callback(cl)
    return mps, pk
