"""Pins for ASAP layering (Sec. II.A) and the cluster partition (Sec. III.A, Eqs. 6-8)."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fig7_partition.txt")


def _read_gold():
    d = {}
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        k, *v = line.split()
        d[k] = v
    return d


def test_fig7_worked_example():
    gold = _read_gold()
    c = synth.fig7_circuit()
    n = int(gold["n_qubits"][0])
    layer, nl = oracle.asap_layers(n, c.gates)
    clusters, stop = oracle.partition(n, c.gates, layer, nl, 0, np.ones(n + 1, np.int64),
                                      int(gold["q_max"][0]), 0, 0)
    want = []
    for tok in gold["clusters"]:
        a, b = (int(x) for x in tok.split("-"))
        want.append((a - 1, b - a + 1))
    assert clusters == want
    assert stop == int(gold["stop_layer"][0])


def test_asap_paper_example():
    # Sec. II.A: after a fully filled 7-layer 8-qubit circuit, U_(6,7) and
    # U_(7,8) appended at the end land in layers 8 and 9.
    b = synth._Builder(8)
    for L in range(7):
        for i in ((0, 2, 4, 6) if L % 2 == 0 else (1, 3, 5)):
            b.g2(synth.CNOT, i, i + 1)
        if L % 2 == 1:
            b.g1(synth.H, 0)
            b.g1(synth.H, 7)
    b.g2(synth.CZ, 5, 6)
    b.g2(synth.CZ, 6, 7)
    c = b.build()
    layer, nl = oracle.asap_layers(8, c.gates)
    assert nl == 9
    assert list(layer[-2:]) == [8, 9]
    # a gate sharing a qubit with the previous one never shares its layer
    b2 = synth._Builder(5)
    b2.g2(synth.CNOT, 2, 3)
    b2.g1(synth.H, 3)
    b2.g1(synth.H, 4)
    layer2, _ = oracle.asap_layers(5, b2.build().gates)
    assert list(layer2) == [1, 2, 1]


def test_eq6_uses_outer_bonds():
    # one CNOT on qubits (2,3) of 6: cluster k=2 bounded by bonds 2 and 4.
    b = synth._Builder(6)
    b.g2(synth.CNOT, 2, 3)
    c = b.build()
    layer, nl = oracle.asap_layers(6, c.gates)
    chi = np.array([1, 2, 4, 8, 4, 2, 1], np.int64)
    # size = 2^2 * chi[2] * chi[4] = 4*4*4 = 64 = 2^6
    assert oracle.partition(6, c.gates, layer, nl, 0, chi, 6, 0, 0) == ([(2, 2)], 1)
    with pytest.raises(RuntimeError):  # 2^6 > 2^5: no layer fits -> error
        oracle.partition(6, c.gates, layer, nl, 0, chi, 5, 0, 0)


def test_lmax_and_kmax():
    c = synth.fig7_circuit()
    layer, nl = oracle.asap_layers(8, c.gates)
    ones = np.ones(9, np.int64)
    cl, stop = oracle.partition(8, c.gates, layer, nl, 0, ones, 30, 1, 0)  # Eq. 8, L_max = 1
    assert stop == 1 and cl == [(0, 2), (2, 2), (4, 2), (6, 2)]
    cl, stop = oracle.partition(8, c.gates, layer, nl, 0, ones, 30, 0, 3)  # k_max = 3
    assert stop == 2
    cl, stop = oracle.partition(8, c.gates, layer, nl, 0, ones, 30, 0, 0)  # unbounded
    assert stop == 5 and cl == [(0, 2), (2, 6)]
    cl, stop = oracle.partition(8, c.gates, layer, nl, 4, ones, 30, 0, 0)  # restart at 4
    assert stop == 5 and cl == [(3, 2)]


def test_non_adjacent_gate_rejected():
    b = synth._Builder(4)
    b.g2(synth.CNOT, 0, 2)
    c = b.build()
    layer, nl = oracle.asap_layers(4, c.gates)
    with pytest.raises(RuntimeError):
        oracle.partition(4, c.gates, layer, nl, 0, np.ones(5, np.int64), 10, 0, 0)


def _brute_properties(n, gates, layer, nl, start, chi, q_max, l_max, k_max, clusters, stop):
    """Eq. 7/8 and maximality, checked by recomputing the bond array by hand."""
    def bond_array(upto):
        bond = np.zeros(n + 1, bool)
        for g, L in zip(gates, layer):
            if start < L <= upto and g[0] > 1:
                lo, hi = min(g[1:1 + g[0]]), max(g[1:1 + g[0]])
                bond[lo + 1:hi + 1] = True
        return bond

    def runs(bond):
        out, b = [], 1
        while b <= n - 1:
            if bond[b]:
                b1 = b
                while b <= n - 1 and bond[b]:
                    b += 1
                out.append((b1 - 1, b - b1 + 1))
            else:
                b += 1
        return out

    def ok(cl):
        return all((k_max <= 0 or k <= k_max) and (2 ** k) * chi[q] * chi[q + k] <= 2 ** q_max
                   for q, k in cl)

    assert runs(bond_array(stop)) == clusters
    assert ok(clusters)
    covered = np.zeros(n, int)
    for q, k in clusters:
        covered[q:q + k] += 1
    assert covered.max(initial=0) <= 1
    if stop < nl and (l_max <= 0 or stop - start < l_max):
        assert not ok(runs(bond_array(stop + 1)))


@pytest.mark.parametrize("seed", range(40))
def test_partition_properties_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(6, 40))
    c = synth.random_structured(n, 12, p1=0.5, p2=float(rng.uniform(0.2, 0.6)),
                                one_q={synth.H: 1.0}, two_q=(synth.CNOT,), seed=seed)
    layer, nl = oracle.asap_layers(n, c.gates)
    chi = np.concatenate([[1], 2 ** rng.integers(0, 5, size=n - 1), [1]]).astype(np.int64)
    q_max = int(rng.integers(10, 20))
    l_max = int(rng.integers(0, 4))
    k_max = int(rng.integers(0, 7))
    if k_max == 1:
        k_max = 2
    start = 0
    while start < nl:
        clusters, stop = oracle.partition(n, c.gates, layer, nl, start, chi, q_max, l_max, k_max)
        assert stop > start
        _brute_properties(n, c.gates, layer, nl, start, chi, q_max, l_max, k_max, clusters, stop)
        start = stop
