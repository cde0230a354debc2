"""Sec. III.B: the virtual MPS of a circuit section (Eq. 9) and the adaptive
grouping of its sites by recursive bipartitioning (Eqs. 10-11).  The oracle is
pinned by hand-derived cases and by Eq. 9's meaning -- an upper bound on the
bond dimensions that the section's gates can create, checked against exact
simulations -- and the library's host functions agree with it exactly."""
import numpy as np
import pytest

import oracle
import synth

P = pytest.importorskip("paper_2502_19289_gb300")


def _hand_circuit():
    b = synth._Builder(6)
    b.g2(synth.CNOT, 0, 1)      # layer 1
    b.g2(synth.CNOT, 2, 3)      # layer 1
    b.g2(synth.CZ, 1, 2)        # layer 2
    b.g2(synth.CNOT, 4, 5)      # layer 1
    b.g2(synth.CNOT, 1, 0)      # layer 3
    return b.build()


def test_virtual_bonds_hand_case():
    c = _hand_circuit()
    layer, nl = oracle.asap_layers(6, c.gates)
    assert list(layer) == [1, 1, 2, 1, 3] and nl == 3
    ones = np.ones(7, dtype=np.int64)
    # all layers: E = [0, 2, 1, 1, 0, 1, 0]; chi~ = min(2^E, 64, 2^min(b, 6-b))
    chi_v, E = oracle.virtual_bonds(6, c.gates, layer, 0, 0, ones, 64)
    assert list(E) == [0, 2, 1, 1, 0, 1, 0]
    assert list(chi_v) == [1, 2, 2, 2, 1, 2, 1]
    # first layer only: E = [0, 1, 0, 1, 0, 1, 0]
    chi_v, E = oracle.virtual_bonds(6, c.gates, layer, 0, 1, ones, 64)
    assert list(E) == [0, 1, 0, 1, 0, 1, 0] and list(chi_v) == [1, 2, 1, 2, 1, 2, 1]
    # layers 2-3 on a state with chi = 3 everywhere inside: 2^E chi capped by chi_max = 5
    chi = np.array([1, 3, 3, 3, 3, 3, 1])
    chi_v, E = oracle.virtual_bonds(6, c.gates, layer, 1, 2, chi, 5)
    assert list(E) == [0, 1, 1, 0, 0, 0, 0] and list(chi_v) == [1, 2, 4, 3, 3, 2, 1]


@pytest.mark.parametrize("seed", range(6))
def test_virtual_bonds_bound_the_exact_bond_dimensions(seed):
    """Gates of operator-Schmidt rank 2 (CNOT, CZ) multiply a bond's Schmidt
    rank by at most 2 each: the exact state after the section never exceeds
    the virtual bond dimensions of Eq. 9 (from |0...0>, chi = 1)."""
    rng = np.random.default_rng(seed)
    n = 10
    c = synth.random_structured(n, 12, p1=0.6, p2=0.4, one_q={synth.H: 0.5, synth.T: 0.5},
                                two_q=(synth.CNOT, synth.CZ), seed=seed)
    layer, nl = oracle.asap_layers(n, c.gates)
    L = int(rng.integers(1, nl + 1))
    keep = layer <= L
    sub = synth.Circuit(n, c.gates[keep], c.params[keep])
    exact = oracle.simulate(sub, 1 << n, 0.0, 2 * n + 2, 0, 0)
    chi_v, _ = oracle.virtual_bonds(n, c.gates, layer, 0, L, np.ones(n + 1, dtype=np.int64), 1 << n)
    assert np.all(exact.chi() <= chi_v), (exact.chi(), chi_v)


def test_grouping_hand_cases():
    # the only bond of dimension 1 in the middle: one cut, two groups of 4
    assert oracle.grouping([1, 2, 4, 8, 1, 8, 4, 2, 1], 6) == [0, 4]
    # 8 qubits with open ends fit Q_max = 8 as one group
    assert oracle.grouping([1, 2, 4, 8, 16, 8, 4, 2, 1], 8) == [0]
    # a product profile halves down to pairs: 8 > 3, cut at 4; 4 > 3, cut at 2 and 6
    assert oracle.grouping([1] * 9, 3) == [0, 2, 4, 6]
    # the cut follows the smallest bond inside the balance window [3, 5]
    assert oracle.grouping([1, 2, 4, 8, 16, 2, 16, 8, 1], 7) == [0, 5]
    # two qubits do not fit Q_max = 1; the only cut leaves a site with a
    # 64-dimensional bond: 1 + 6 > 1, no grouping exists
    with pytest.raises(ValueError):
        oracle.grouping([1, 64, 1], 1)
    # three qubits with open ends fit Q_max = 5 whatever the inner bonds
    assert oracle.grouping([1, 64, 64, 1], 5) == [0]


def test_grouping_properties_random():
    rng = np.random.default_rng(3)
    for _ in range(300):
        n = int(rng.integers(1, 40))
        chi_v = np.concatenate([[1], 2 ** rng.integers(0, 6, n - 1), [1]]) if n > 1 else np.array([1, 1])
        q_max = int(rng.integers(12, 30))
        starts = oracle.grouping(chi_v, q_max)
        ends = starts[1:] + [n]
        assert starts[0] == 0 and all(a < b for a, b in zip(starts, ends))
        for lo, hi in zip(starts, ends):
            bl = 1 if lo == 0 else int(chi_v[lo])
            br = 1 if hi == n else int(chi_v[hi])
            assert (hi - lo) + np.log2(bl) + np.log2(br) <= q_max + 1e-12


def test_library_matches_oracle():
    rng = np.random.default_rng(9)
    for seed in range(200):
        n = int(rng.integers(2, 48))
        c = synth.random_structured(n, int(rng.integers(2, 30)), p1=0.5, p2=float(rng.uniform(0.1, 0.7)),
                                    one_q={synth.H: 1.0}, two_q=(synth.CNOT, synth.CZ, synth.SWAP), seed=seed)
        circ = P.Circuit(n, c.gates, c.params)
        layer, nl = oracle.asap_layers(n, c.gates)
        chi = np.concatenate([[1], 2 ** rng.integers(0, 5, n - 1), [1]]).astype(np.int64)
        start = int(rng.integers(0, max(nl, 1)))
        l_max = int(rng.choice([0, 1, 3, 7]))
        chi_max = int(2 ** rng.integers(2, 12))
        want, E = oracle.virtual_bonds(n, c.gates, layer, start, l_max, chi, chi_max)
        got, Eg = P.virtual_mps_bonds(circ.gates, circ.n_gates, n, start, l_max, chi, chi_max)
        np.testing.assert_array_equal(got, want)
        np.testing.assert_array_equal(Eg, E)
        q_max = int(rng.integers(2 + 2 * int(np.log2(chi_max)), 34))
        try:
            ref = oracle.grouping(want, q_max)
        except ValueError:
            with pytest.raises(P.CtebdError, match="does not fit"):
                P.adaptive_grouping(got, q_max)
            continue
        assert list(P.adaptive_grouping(got, q_max)) == ref
