"""GPU: packed independent circuits (clusters of all circuits in the same
launches, every circuit with its own stop layer) and standard TEBD (L_max = 1,
k_max = 2) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib, statevector_of

pytestmark = pytest.mark.gpu


def test_packed_circuits_match_their_own_runs():
    P = lib()
    rng = np.random.default_rng(5)
    circs = []
    for i in range(5):
        n = int(rng.integers(6, 11))
        t = float(rng.uniform(0.05, 0.25))
        c = synth.random_structured(n, int(rng.integers(10, 25)), p1=0.7, p2=0.4,
                                    one_q={synth.T: t, synth.H: (1 - t) / 2, synth.S: (1 - t) / 2},
                                    two_q=(synth.CNOT, synth.CZ), seed=100 + i)
        circs.append(c)
    k_max, chi, cut = 4, 16, 1e-12
    q_max = k_max + 2 * 4
    cfg = P.make_config(1, chi, cut, q_max, 0, k_max, P.FP64)
    mps, pk = P.simulate_packed([(c.n_qubits, c.gates, c.params) for c in circs], cfg)
    chis = mps.bond_dims()
    for c, off in zip(circs, pk.offsets):
        n = c.n_qubits
        assert chis[off] == 1 and chis[off + n] == 1          # circuits never entangle
        ref = oracle.simulate(c, chi, cut, q_max, 0, k_max)
        assert list(chis[off:off + n + 1]) == list(ref.chi())
        sites = [mps.site(off + q) for q in range(n)]
        sv = statevector_of(sites)
        np.testing.assert_allclose(sv, ref.statevector(), atol=1e-10)


def test_standard_tebd_on_gpu():
    P = lib()
    w = synth.WORKLOADS[1]
    c = w.circuit(2, 1)
    circ = P.Circuit(c.n_qubits, c.gates, c.params)
    cfg = P.make_config(12, 64, 0.0, 16, 1, 2, P.FP64)            # one layer, one gate per split
    steps = []
    mps = P.simulate(circ, cfg, callback=lambda s, e, cl, f: steps.append(e - s))
    assert set(steps) == {1}
    psi = oracle.statevector(c)
    np.testing.assert_allclose(statevector_of([mps.site(q) for q in range(12)]), psi, atol=1e-12)


def test_packed_cfg5_shape_truncated_fp32():
    """The packed configuration's statistics at a size the oracle finishes: 12
    independent Clifford+T circuits (n ~ U[16, 28], 40-100 layers, T density
    ~ U[5%, 25%]) packed into the same batched launches in FP32 with
    truncation; every circuit against its own oracle run (bond dimensions,
    fidelity product of its splits, normalised state overlap)."""
    P = lib()
    from gpu_helpers import fidelity_overlap
    rng = np.random.default_rng(55)
    circs = []
    for i in range(12):
        n = int(rng.integers(16, 29))
        t = float(rng.uniform(0.05, 0.25))
        circs.append(synth.random_structured(n, int(rng.integers(40, 101)), p1=0.5, p2=0.3,
                                             one_q={synth.T: t, synth.H: (1 - t) / 2, synth.S: (1 - t) / 2},
                                             two_q=(synth.CNOT, synth.CZ), seed=5500 + i))
    k_max, chi, cut = 4, 16, 1e-8
    q_max = k_max + 2 * 4
    cfg = P.make_config(1, chi, cut, q_max, 0, k_max, P.FP32)
    mps, pk = P.simulate_packed([(c.n_qubits, c.gates, c.params) for c in circs], cfg)
    chis = mps.bond_dims()
    truncated, logF = 0, 0.0
    for c, off in zip(circs, pk.offsets):
        n = c.n_qubits
        ref = oracle.simulate(c, chi, cut, q_max, 0, k_max, floor=1e-6)
        assert list(chis[off:off + n + 1]) == list(ref.chi())
        truncated += ref.logF < -1e-6
        logF += ref.logF
        sites = [mps.site(off + q) for q in range(n)]
        lams = [mps.lam(off + b) for b in range(n + 1)]
        got = oracle.MPS.from_arrays(sites, lams)
        assert fidelity_overlap(ref, got) >= 1 - 1e-6
    assert truncated >= 3
    # the packed run's fidelity product is the product over the circuits (Eq. 5)
    assert abs(np.log(mps.fidelity()) - logF) <= 1e-5 * max(1.0, abs(logF))
