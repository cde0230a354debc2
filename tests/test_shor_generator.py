"""CPU: Shor's order-finding circuit in Beauregard's construction (Sec. IV.B),
pinned by number theory rather than by the oracle's own arithmetic:

* N = 15, a = 7 (order 4), 3 counting qubits: the counting register is
  exactly uniform over the multiples of 2^t / 4, the work register is uniform
  over the powers of 7 mod 15, and the addition register and the ancilla end
  in |0> (a dropped phase, a wrong modular constant or a missing ancilla reset
  breaks one of these);
* N = 21, a = 2 (order 6, not a power of two): the whole counting
  distribution equals its closed form
  P(y) = sum_z |2^-t sum_{C : a^C = z mod N} exp(-2 pi i y C / 2^t)|^2;
* every two-qubit gate acts on neighbours, as in the paper's SWAP routing;
* the qubit counts of the paper's five instances (reading G18);
* the oracle's cluster-TEBD reproduces the state vector on the N = 15 circuit."""
import math

import numpy as np
import pytest

import oracle
from synth.shor import counting_qubits, shor_circuit, shor_registers


def _marginal(psi, n, qubits):
    p = np.abs(psi.reshape((2,) * n)) ** 2
    return p.sum(axis=tuple(i for i in range(n) if i not in qubits))


def _counting_distribution(psi, n, t):
    """P(y) with y's bit k read from counting qubit t - 1 - k."""
    pc = _marginal(psi, n, list(range(t)))
    out = np.zeros(1 << t)
    for idx in np.ndindex(*(2,) * t):
        out[sum(idx[t - 1 - k] << k for k in range(t))] += pc[idx]
    return out


@pytest.fixture(scope="module")
def n15():
    c = shor_circuit(15, 7, 3)
    return c, oracle.statevector(c)


def test_order_four_gives_exact_peaks(n15):
    c, psi = n15
    t = 3
    assert c.n_qubits == t + 2 * 4 + 2
    P = _counting_distribution(psi, c.n_qubits, t)
    expect = np.zeros(8)
    expect[[0, 2, 4, 6]] = 0.25
    np.testing.assert_allclose(P, expect, atol=1e-10)


def test_work_register_and_ancillas(n15):
    c, psi = n15
    R = shor_registers(15, 3)
    pb = _marginal(psi, c.n_qubits, R["b"] + [R["anc"]]).reshape(-1)
    assert pb[0] == pytest.approx(1.0, abs=1e-10)
    px = _marginal(psi, c.n_qubits, R["x"])
    vals = {}
    for idx in np.ndindex(*(2,) * len(R["x"])):
        v = sum(idx[k] << k for k in range(len(R["x"])))   # x_0 least significant
        if px[idx] > 1e-12:
            vals[v] = px[idx]
    assert sorted(vals) == sorted({pow(7, k, 15) for k in range(4)})
    np.testing.assert_allclose(list(vals.values()), 0.25, atol=1e-10)


def test_order_six_matches_closed_form():
    N, a, t = 21, 2, 3
    c = shor_circuit(N, a, t)
    psi = oracle.statevector(c)
    P = _counting_distribution(psi, c.n_qubits, t)
    C = np.arange(1 << t)
    z = np.array([pow(a, int(k), N) for k in C])
    ref = np.zeros(1 << t)
    for y in range(1 << t):
        ph = np.exp(-2j * np.pi * y * C / (1 << t))
        ref[y] = sum(abs(ph[z == v].sum() / (1 << t)) ** 2 for v in np.unique(z))
    assert ref.sum() == pytest.approx(1.0)
    np.testing.assert_allclose(P, ref, atol=1e-10)


def test_nearest_neighbour_gates_only(n15):
    c, _ = n15
    g = c.gates
    two = g[g[:, 0] == 2]
    assert len(two) > 0 and np.all(np.abs(two[:, 1] - two[:, 2]) == 1)
    assert not np.any(g[:, 0] == 3)


def test_qubit_counts_of_the_paper_instances():
    # (N, eps, qubits the paper reports) for its five factoring instances;
    # this construction uses t + 2n + 2 qubits, one fewer (reading G18)
    for N, eps, qubits in ((15, 1e-3, 29), (21, 1e-4, 37), (35, 1e-5, 44), (91, 1e-5, 48), (221, 1e-9, 65)):
        n = math.ceil(math.log2(N))
        t = counting_qubits(N, eps)
        assert t + 2 * n + 3 == qubits
    c = shor_circuit(15, 7, 2)
    assert c.n_qubits == 2 + 2 * 4 + 2


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        shor_circuit(15, 5, 2)      # gcd(5, 15) = 5
    with pytest.raises(ValueError):
        shor_circuit(15, 1, 2)
    with pytest.raises(ValueError):
        shor_circuit(15, 7, 0)
    with pytest.raises(ValueError):
        counting_qubits(15, 0.0)


def test_cluster_tebd_oracle_reproduces_state(n15):
    """The oracle's cluster-TEBD (clusters of up to 8 qubits over as many
    layers as Eq. 7 allows) on the N = 15 circuit, against the state vector."""
    c, psi = n15
    m = oracle.simulate(c, chi_max=64, cutoff=0.0, q_max=3 + 12, l_max=0, k_max=8)
    sv = m.statevector()
    assert abs(np.vdot(sv, psi)) / np.linalg.norm(sv) >= 1 - 1e-10
    assert m.logF == pytest.approx(0.0, abs=1e-12)
