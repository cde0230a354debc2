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
* the oracle's cluster-TEBD and standard TEBD reproduce the state vector on
  the N = 15 circuit.  The long standard-TEBD run (13 548 iterations) also
  pins the oracle's one-sided Jacobi SVD on rank-deficient splits: a SWAP
  split there produces columns of subnormal norm."""
import math

import numpy as np
import pytest

import oracle
from synth.shor import counting_qubits, shor_build, shor_circuit, shor_registers


def _bits_distribution(psi, n, positions, weights):
    """Distribution of sum_j weights[j] * (bit at chain position positions[j])."""
    p = np.abs(psi.reshape((2,) * n)) ** 2
    pm = p.sum(axis=tuple(i for i in range(n) if i not in positions))
    axes = sorted(positions)                       # pm's axes follow the chain order
    out = {}
    for idx in np.ndindex(*(2,) * len(axes)):
        bit = dict(zip(axes, idx))
        v = sum(w * bit[q] for q, w in zip(positions, weights))
        out[v] = out.get(v, 0.0) + pm[idx]
    return out


def _counting_distribution(psi, n, cpos):
    """P(y), y's bit k read from counting qubit c_(t-1-k) (at chain position
    cpos[t-1-k])."""
    t = len(cpos)
    d = _bits_distribution(psi, n, cpos, [1 << (t - 1 - j) for j in range(t)])
    return np.array([d.get(y, 0.0) for y in range(1 << t)])


def _marginal(psi, n, qubits):
    p = np.abs(psi.reshape((2,) * n)) ** 2
    return p.sum(axis=tuple(i for i in range(n) if i not in qubits))


@pytest.fixture(scope="module")
def n15():
    c = shor_circuit(15, 7, 3)
    return c, oracle.statevector(c)


@pytest.fixture(scope="module", params=["return", "lazy"])
def n15_routed(request):
    c, regs = shor_build(15, 7, 3, routing=request.param)
    return c, regs, oracle.statevector(c)


def test_order_four_gives_exact_peaks(n15_routed):
    c, regs, psi = n15_routed
    t = 3
    assert c.n_qubits == t + 2 * 4 + 2
    P = _counting_distribution(psi, c.n_qubits, regs["c"])
    expect = np.zeros(8)
    expect[[0, 2, 4, 6]] = 0.25
    np.testing.assert_allclose(P, expect, atol=1e-10)


def test_work_register_and_ancillas(n15_routed):
    c, regs, psi = n15_routed
    n = c.n_qubits
    zero = _bits_distribution(psi, n, regs["b"] + [regs["anc"]], [1 << k for k in range(len(regs["b"]) + 1)])
    assert zero.get(0, 0.0) == pytest.approx(1.0, abs=1e-10)
    x = _bits_distribution(psi, n, regs["x"], [1 << k for k in range(len(regs["x"]))])
    vals = {v: p for v, p in x.items() if p > 1e-12}
    assert sorted(vals) == sorted({pow(7, k, 15) for k in range(4)})
    np.testing.assert_allclose(list(vals.values()), 0.25, atol=1e-10)


def test_return_routing_keeps_chain_order():
    _, regs = shor_build(15, 7, 3)
    assert regs == shor_registers(15, 3)


@pytest.mark.parametrize("routing", ["return", "lazy"])
def test_order_six_matches_closed_form(routing):
    N, a, t = 21, 2, 3
    c, regs = shor_build(N, a, t, routing=routing)
    psi = oracle.statevector(c)
    P = _counting_distribution(psi, c.n_qubits, regs["c"])
    C = np.arange(1 << t)
    z = np.array([pow(a, int(k), N) for k in C])
    ref = np.zeros(1 << t)
    for y in range(1 << t):
        ph = np.exp(-2j * np.pi * y * C / (1 << t))
        ref[y] = sum(abs(ph[z == v].sum() / (1 << t)) ** 2 for v in np.unique(z))
    assert ref.sum() == pytest.approx(1.0)
    np.testing.assert_allclose(P, ref, atol=1e-10)


def test_nearest_neighbour_gates_only(n15_routed):
    c, _, _ = n15_routed
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
    with pytest.raises(ValueError):
        shor_build(15, 7, 2, routing="greedy")


def test_cluster_tebd_oracle_reproduces_state(n15):
    """The oracle's cluster-TEBD (clusters of up to 8 qubits over as many
    layers as Eq. 7 allows) on the N = 15 circuit, against the state vector."""
    c, psi = n15
    m = oracle.simulate(c, chi_max=64, cutoff=0.0, q_max=3 + 12, l_max=0, k_max=8)
    sv = m.statevector()
    assert abs(np.vdot(sv, psi)) / np.linalg.norm(sv) >= 1 - 1e-10
    assert m.logF == pytest.approx(0.0, abs=1e-12)


def test_standard_tebd_oracle_reproduces_state(n15):
    """Standard TEBD (one layer per iteration, two-qubit clusters) over all
    13 548 layers of the N = 15 circuit."""
    c, psi = n15
    m = oracle.simulate(c, chi_max=64, cutoff=0.0, q_max=2 + 12, l_max=1, k_max=2)
    sv = m.statevector()
    assert abs(np.vdot(sv, psi)) / np.linalg.norm(sv) >= 1 - 1e-10
    assert max(m.chi()) <= 4


def test_oracle_svd_rank_deficient_split(n15):
    """The split of the SWAP in layer 4380 of the N = 15 circuit (standard
    TEBD): a 4 x 4 Schmidt-weighted matrix of rank 2.  Its singular values
    against numpy's, and the right singular vectors orthonormal."""
    c, _ = n15
    layer, _ = oracle.asap_layers(c.n_qubits, c.gates)
    sel = layer <= 4379
    import synth
    sub = synth.Circuit(c.n_qubits, c.gates[sel], c.params[sel])
    m = oracle.simulate(sub, chi_max=64, cutoff=0.0, q_max=2 + 12, l_max=1, k_max=2)
    swap = [(g, p) for g, p in zip(c.gates[layer == 4380], c.params[layer == 4380])]
    assert len(swap) == 1 and swap[0][0][4] == synth.SWAP
    q = int(min(swap[0][0][1], swap[0][0][2]))
    th = np.einsum("asb,btc->astc", m.site(q), m.site(q + 1))
    th = np.einsum("stuv,auvc->astc", oracle.gate_matrix(synth.SWAP).reshape(2, 2, 2, 2), th)
    lam = m.lam(q)
    M = (lam[:, None, None, None] * th).reshape(th.shape[0] * 2, -1)
    s = np.zeros(min(M.shape))
    Y = np.zeros(2 * M.shape[1] * len(s))
    oracle._check(oracle._L().orc_svd(M.shape[0], M.shape[1], oracle._c128(M).reshape(-1), s, Y))
    Y = Y.view(np.complex128).reshape(M.shape[1], len(s))
    np.testing.assert_allclose(s, np.linalg.svd(M, compute_uv=False), atol=1e-14)
    np.testing.assert_allclose(Y.conj().T @ Y, np.eye(len(s)), atol=1e-13)


def test_oracle_rejects_zero_floor(n15):
    c, _ = n15
    with pytest.raises(ValueError):
        oracle.simulate(c, chi_max=64, cutoff=0.0, q_max=14, l_max=1, k_max=2, floor=0.0)
