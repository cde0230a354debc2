"""CPU checks of the C ABI: the library loads, exports every entry point that
include/ctebd.h declares, and its host-side pieces (Sec. II.A layering,
Sec. III.A partition, cluster unitaries) agree bit-exactly with the oracle's
independent implementation.  No GPU compute is called here."""
import os
import re

import numpy as np
import pytest

import oracle
import synth

P = pytest.importorskip("paper_2502_19289_gb300")
HDR = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "ctebd.h")


def _declared():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*int\s+(\w+)\s*\(", txt, flags=re.M)))


def test_every_declared_symbol_is_exported():
    names = _declared()
    assert {"mps_create", "cluster_partition", "apply_cluster", "truncate_split", "fidelity",
            "amplitude", "step"} <= set(names)
    for n in names:
        assert hasattr(P.lib, n), n


def test_create_without_gpu_fails_loudly():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("GPU present")
    except ImportError:
        pass
    cfg = P.make_config(4, 8, 0.0, 8, 0, 4, P.FP64)
    with pytest.raises(P.CtebdError, match="CUDA|device"):
        P.MPS(cfg)


def test_config_preconditions_rejected():
    with pytest.raises(P.CtebdError, match="q_max"):
        P.MPS(P.make_config(4, 64, 0.0, 10, 0, 4, P.FP64))   # q_max < 2 + 2 log2 64
    with pytest.raises(P.CtebdError, match="k_max"):
        P.MPS(P.make_config(4, 8, 0.0, 20, 0, 1, P.FP64))


def _layers_both(c):
    circ = P.Circuit(c.n_qubits, c.gates, c.params)
    lo, nlo = oracle.asap_layers(c.n_qubits, c.gates)
    mine = np.array([circ.gates[i].layer for i in range(circ.n_gates)])
    return circ, lo, nlo, mine


@pytest.mark.parametrize("cfg_id", [1, 2, 3])
def test_layers_match_oracle(cfg_id):
    w = synth.reduced(cfg_id, 30, 20)
    c = w.circuit(3, cfg_id)
    circ, lo, nlo, mine = _layers_both(c)
    assert circ.n_layers == nlo
    np.testing.assert_array_equal(mine, lo)


def test_partition_bit_exact_random():
    rng = np.random.default_rng(123)
    n_cases = 0
    for seed in range(300):
        n = int(rng.integers(4, 60))
        c = synth.random_structured(n, int(rng.integers(3, 25)), p1=0.5,
                                    p2=float(rng.uniform(0.1, 0.7)),
                                    one_q={synth.H: 1.0}, two_q=(synth.CNOT, synth.CZ),
                                    long_range_frac=0.1, seed=seed)
        circ, lo, nlo, _ = _layers_both(c)
        k_max = int(rng.choice([0, 2, 3, 4, 6, 8]))
        l_max = int(rng.choice([0, 0, 1, 2, 5]))
        chi_max_lg = int(rng.integers(0, 6))
        q_max = 2 + 2 * chi_max_lg + int(rng.integers(0, 8))
        cfg = P.make_config(n, 1 << chi_max_lg, 0.0, q_max, l_max, k_max)
        for _ in range(4):
            chi = np.concatenate([[1], 2 ** rng.integers(0, chi_max_lg + 1, n - 1), [1]])
            start = int(rng.integers(0, max(nlo, 1)))
            want = oracle.partition(n, c.gates, lo, nlo, start, chi.astype(np.int64), q_max,
                                    l_max, k_max)
            got, stop = P.cluster_partition(circ.gates, circ.n_gates, start, chi, cfg)
            assert [(x.q0, x.k) for x in got] == want[0]
            assert stop == want[1]
            assert all(x.layer_lo == start and x.layer_hi == stop for x in got)
            n_cases += 1
    assert n_cases == 1200


def test_partition_fig7():
    c = synth.fig7_circuit()
    circ = P.Circuit(8, c.gates, c.params)
    cfg = P.make_config(8, 1, 0.0, 5, 0, 0)
    got, stop = P.cluster_partition(circ.gates, circ.n_gates, 0, np.ones(9), cfg)
    assert [(x.q0, x.k) for x in got] == [(0, 2), (2, 2), (4, 4)] and stop == 4


def test_partition_errors():
    b = synth._Builder(4)
    b.g2(synth.CNOT, 0, 2)
    c = b.build()
    circ = P.Circuit(4, c.gates, c.params)
    with pytest.raises(P.CtebdError, match="adjacent"):
        P.cluster_partition(circ.gates, circ.n_gates, 0, np.ones(5), P.make_config(4, 1, 0, 10))


@pytest.mark.parametrize("seed", range(6))
def test_cluster_unitary_matches_oracle(seed):
    w = synth.reduced(2, 16, 12)
    c = w.circuit(seed, 2)
    circ, lo, nlo, _ = _layers_both(c)
    cfg = P.make_config(16, 1, 0.0, 64, 0, 8)
    clusters, stop = P.cluster_partition(circ.gates, circ.n_gates, 0, np.ones(17), cfg)
    assert clusters
    for cl in clusters:
        U = P.cluster_unitary(circ.gates, circ.n_gates, cl)
        Uo = oracle.cluster_unitary(cl.q0, cl.k, c, lo, 0, stop)
        np.testing.assert_allclose(U, Uo, atol=1e-14)


@pytest.mark.parametrize("source", ["paper-nonclifford", "shor"])
def test_cluster_unitary_all_gate_kinds(source):
    """Cluster unitaries of 6 to 10 qubits over every gate kind: permutation
    gates (X, CNOT, SWAP), diagonal ones (Z, S, T, P, CZ, CS, CT, CP) and dense
    ones (H, Y, X^1/4, sqrt W, CY, CH, sqrt SWAP), against the oracle's product
    and against unitarity."""
    if source == "shor":
        from synth.shor import shor_circuit
        c = shor_circuit(15, 7, 2)
    else:
        c = synth.paper_random_structured(14, 12, clifford=False, seed=21)
    n = c.n_qubits
    circ, lo, nlo, _ = _layers_both(c)
    kmax = 8 if source == "shor" else 10
    cfg = P.make_config(n, 1, 0.0, kmax, 0, kmax)
    start, seen, kseen = 0, 0, 0
    while start < circ.n_layers and seen < 16:
        clusters, stop = P.cluster_partition(circ.gates, circ.n_gates, start, np.ones(n + 1), cfg)
        for cl in clusters:
            U = P.cluster_unitary(circ.gates, circ.n_gates, cl)
            Uo = oracle.cluster_unitary(cl.q0, cl.k, c, lo, start, stop)
            np.testing.assert_allclose(U, Uo, atol=1e-13)
            np.testing.assert_allclose(U @ U.conj().T, np.eye(U.shape[0]), atol=1e-12)
            seen += 1
            kseen = max(kseen, cl.k)
        start = stop
    assert kseen >= 6


@pytest.mark.parametrize("source", ["cfg2", "shor"])
def test_layer_sorted_copy(source):
    """Circuit.gates_by_layer holds the same gates in non-decreasing layer
    order (the given order within a layer), and the partition and the
    cluster unitaries it feeds are those of the given order."""
    if source == "shor":
        from synth.shor import shor_circuit
        c = shor_circuit(15, 7, 2)
    else:
        c = synth.reduced(2, 24, 20).circuit(2, 2)
    n = c.n_qubits
    circ = P.Circuit(n, c.gates, c.params)
    g0, g1 = circ.gates, circ.gates_by_layer
    rows = lambda g, i: (g[i].layer, g[i].n_q, tuple(g[i].q), g[i].kind, g[i].param)
    a = [rows(g0, i) for i in range(circ.n_gates)]
    b = [rows(g1, i) for i in range(circ.n_gates)]
    assert [x[0] for x in b] == sorted(x[0] for x in b)
    assert b == sorted(a, key=lambda x: x[0])          # stable: Python's sort is stable
    chis = np.minimum(np.asarray([2 ** min(q, n - q) for q in range(n + 1)], dtype=np.int32), 8)
    for cfg in (P.make_config(n, 64, 1e-8, 8, 1, 2), P.make_config(n, 64, 1e-8, 12, 0, 6)):
        start = 0
        while start < circ.n_layers:
            cl0, s0 = P.cluster_partition(g0, circ.n_gates, start, chis, cfg)
            cl1, s1 = P.cluster_partition(g1, circ.n_gates, start, chis, cfg)
            assert s0 == s1 and [(x.q0, x.k) for x in cl0] == [(x.q0, x.k) for x in cl1]
            for x, y in zip(cl0, cl1):
                np.testing.assert_array_equal(P.cluster_unitary(g0, circ.n_gates, x),
                                              P.cluster_unitary(g1, circ.n_gates, y))
            start = s0
