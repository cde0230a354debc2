"""The paper's random-structured circuits (Sec. IV.A): every slot of every
layer filled with a one- or two-qubit gate (p = 0.5), Clifford and
non-Clifford gate sets (App. A).  CPU checks: the generator's statistics and
gate sets, the library's host partition and cluster unitaries against the
oracle on these circuits (every App. A gate, both control orientations), and
the oracle's MPS against its state vector and, for the Clifford family, the
stabilizer tableau."""
import numpy as np
import pytest

import oracle
import synth

P = pytest.importorskip("paper_2502_19289_gb300")


def test_slot_filling_and_gate_sets():
    for clifford in (True, False):
        c = synth.paper_random_structured(40, 30, clifford=clifford, seed=5)
        g = c.gates
        one, two = g[g[:, 0] == 1], g[g[:, 0] == 2]
        # every layer fills every qubit once: n slots per layer
        assert len(one) + 2 * len(two) == 40 * 30
        allowed1 = {k for k, _ in (synth.PAPER_CLIFFORD_1Q if clifford else synth.PAPER_NONCLIFFORD_1Q)}
        allowed2 = set(synth.PAPER_CLIFFORD_2Q if clifford else synth.PAPER_NONCLIFFORD_2Q)
        assert set(one[:, 4]) == allowed1 and set(two[:, 4]) == allowed2
        assert np.all(np.abs(two[:, 1] - two[:, 2]) == 1)            # nearest neighbours
        assert 0.3 < np.mean(two[:, 1] < two[:, 2]) < 0.7             # both orientations
        # every slot decision places one gate, a two-qubit one with p = 0.5 (the
        # last qubit of a layer can only take a one-qubit gate)
        share = len(two) / (len(one) + len(two))
        assert 0.44 < share < 0.54, share
        # ASAP layering reproduces the generation layers (every layer is full)
        layer, nl = oracle.asap_layers(40, c.gates)
        assert nl == 30
        if not clifford:
            pk = c.params[g[:, 4] == synth.P]
            assert len(pk) and np.allclose(pk, 0.75 * np.pi)


@pytest.mark.parametrize("seed", range(4))
def test_host_partition_and_unitaries_match_oracle(seed):
    c = synth.paper_random_structured(14, 8, clifford=seed % 2 == 0, seed=seed)
    circ = P.Circuit(14, c.gates, c.params)
    lo, nlo = oracle.asap_layers(14, c.gates)
    assert circ.n_layers == nlo
    chi = np.ones(15, dtype=np.int64)
    for q_max, k_max in ((10, 4), (14, 8), (8, 3)):
        cfg = P.make_config(14, 1, 0.0, q_max, 0, k_max)
        want = oracle.partition(14, c.gates, lo, nlo, 0, chi, q_max, 0, k_max)
        got, stop = P.cluster_partition(circ.gates, circ.n_gates, 0, chi, cfg)
        assert [(x.q0, x.k) for x in got] == want[0] and stop == want[1]
        for cl in got:
            U = P.cluster_unitary(circ.gates, circ.n_gates, cl)
            Uo = oracle.cluster_unitary(cl.q0, cl.k, c, lo, 0, stop)
            np.testing.assert_allclose(U, Uo, atol=1e-13)
            np.testing.assert_allclose(U @ U.conj().T, np.eye(len(U)), atol=1e-12)


@pytest.mark.parametrize("clifford", [True, False])
def test_oracle_mps_equals_statevector(clifford):
    c = synth.paper_random_structured(10, 12, clifford=clifford, seed=7)
    m = oracle.simulate(c, 32, 0.0, 4 + 10, 0, 4)
    psi = oracle.statevector(c)
    np.testing.assert_allclose(m.statevector(), psi, atol=1e-12)
    if clifford:   # flat spectra, chi_b = 2^S_b (Gottesman-Knill)
        S = oracle.stabilizer_entropies(c)
        assert list(m.chi()) == [int(2 ** s) for s in S]
