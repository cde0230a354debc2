"""GPU: the eigen-solve sweep loop run on the device (one CUDA graph with a
WHILE node per batched eigen-solve) against the same sweeps launched round by
round from the host.  Same kernels in the same order: equal bond dimensions
and sweep counts, fidelities equal to rounding, and both match the oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import as_oracle, fidelity_overlap, lib

pytestmark = pytest.mark.gpu


def _run(P, c, w, chi, graphs, precision):
    P.set_sweep_graphs(2 if graphs else 0)
    try:
        circ = P.Circuit(c.n_qubits, c.gates, c.params)
        cfg = P.make_config(c.n_qubits, chi, w.cutoff, w.q_max, 0, w.k_max, precision)
        mps = P.MPS(cfg)
        start, logs = 0, []
        while start < circ.n_layers:
            clusters, stop, f = P.run_iteration(mps, circ, start)
            if clusters:
                logs.append(mps.split_log())
            start = stop
        return mps, np.concatenate(logs)
    finally:
        P.set_sweep_graphs(1)


@pytest.mark.parametrize("precision_name,chi", [("FP32", 32), ("FP32", 256), ("FP64", 32)])
def test_device_sweeps_match_host_sweeps(precision_name, chi):
    P = lib()
    precision = getattr(P, precision_name)
    w = synth.reduced(2, 20, 110)
    c = w.circuit(0, 2)
    m_g, log_g = _run(P, c, w, chi, True, precision)
    m_h, log_h = _run(P, c, w, chi, False, precision)
    assert list(m_g.bond_dims()) == list(m_h.bond_dims())
    np.testing.assert_array_equal(log_g[:, 5], log_h[:, 5])            # ranks
    diff = np.nonzero(np.any(log_g[:, 12:14] != log_h[:, 12:14], axis=1))[0]
    assert len(diff) == 0, [(int(i), log_g[i, [0, 1, 2, 4, 12, 13]].tolist(), log_h[i, 12:14].tolist())
                            for i in diff[:8]]   # sweeps of both passes: (row, [q0, k, bond, n, sw1, sw2], host)
    np.testing.assert_allclose(log_g[:, 6], log_h[:, 6], rtol=1e-9)     # per-split f
    assert abs(m_g.fidelity() / m_h.fidelity() - 1) <= 1e-9
    ref = oracle.simulate(c, chi, w.cutoff, w.q_max, 0, w.k_max)
    assert fidelity_overlap(ref, as_oracle(m_g)) >= 1 - 1e-6
    assert abs(m_g.fidelity() / np.exp(ref.logF) - 1) <= 1e-5


def test_switch_rejects_other_values():
    P = lib()
    import ctypes
    assert P._lib.ctebd_set_sweep_graphs(ctypes.c_int(3)) != 0
    assert P._lib.ctebd_set_sweep_graphs(ctypes.c_int(-1)) != 0



def test_compact_tail_matches_host_sweeps():
    """A batch of more than eight problems with some at least 32 blocks wide
    runs its last sweeps on a compact chain (IF nodes in the device-side
    loop).  One iteration of the chi_max = 1024 workload's circuit on 40
    qubits saturated at chi = 512 (11 two-qubit clusters, 1024-wide splits):
    both loops give the same ranks, sweep counts and fidelities, bit for bit."""
    P = lib()
    n, chi = 40, 512
    w = synth.WORKLOADS[4]
    c = synth.random_structured(n, w.n_layers, p1=w.p1, p2=w.p2, one_q=w.one_q,
                                two_q=w.two_q, seed=4000)
    circ = P.Circuit(n, c.gates, c.params)
    chis, sites, lams = synth.random_right_canonical(n, chi, seed=4001, dtype=np.complex64)
    cfg = P.make_config(n, chi, w.cutoff, w.k_max + 2 * 9, 0, w.k_max, P.FP32)
    out = []
    for graphs in (True, False):
        P.set_sweep_graphs(2 if graphs else 0)
        try:
            mps = P.MPS(cfg)
            mps.load(chis, sites, lams)
            clusters, _, f = P.run_iteration(mps, circ, 0)
            out.append((len(clusters), list(mps.bond_dims()), mps.split_log(), np.asarray(f)))
        finally:
            P.set_sweep_graphs(1)
    (nc, chi_g, log_g, f_g), (_, chi_h, log_h, f_h) = out
    assert nc > 8 and int(np.sum(log_g[:, 4] >= 1024)) > 0, (nc, log_g[:, 4].tolist())
    assert chi_g == chi_h
    np.testing.assert_array_equal(log_g[:, [5, 12, 13]], log_h[:, [5, 12, 13]])   # ranks, sweeps
    np.testing.assert_array_equal(f_g, f_h)
