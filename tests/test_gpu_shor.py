"""GPU: cluster-TEBD through the library on Shor's order-finding circuit
(Sec. IV.B; Beauregard's construction routed to nearest neighbours), N = 15,
a = 7, 3 counting qubits: 13 qubits, 16 296 gates in 13 548 sparse layers,
contracted in 847 cluster-TEBD iterations.  The final state against the
oracle's state vector, and the counting register against its exact peaks."""
import numpy as np
import pytest

import oracle
from gpu_helpers import lib, statevector_of
from synth.shor import shor_circuit

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def n15():
    c = shor_circuit(15, 7, 3)
    return c, oracle.statevector(c)


@pytest.mark.parametrize("precision_name,cutoff,tol", [("FP32", 1e-8, 1e-5), ("FP64", 1e-12, 1e-10)])
def test_shor_n15_cluster_tebd(n15, precision_name, cutoff, tol):
    P = lib()
    c, psi = n15
    n, t = c.n_qubits, 3
    cfg = P.make_config(n, 64, cutoff, 3 + 12, 0, 8, getattr(P, precision_name))
    iters = []
    mps = P.simulate(P.Circuit(n, c.gates, c.params), cfg, callback=lambda s, e, cl, f: iters.append(len(cl)))
    assert len(iters) < 1000            # many layers per iteration (13 548 layers)
    assert max(mps.bond_dims()) <= 16
    sv = statevector_of([mps.site(q) for q in range(n)])
    assert abs(np.vdot(sv, psi)) / np.linalg.norm(sv) >= 1 - tol
    assert abs(mps.fidelity() - 1) <= tol
    p = np.abs(sv.reshape((2,) * n)) ** 2
    pc = p.sum(axis=tuple(range(t, n)))
    P_y = np.zeros(8)
    for idx in np.ndindex(2, 2, 2):
        P_y[sum(idx[t - 1 - k] << k for k in range(t))] += pc[idx]
    expect = np.zeros(8)
    expect[[0, 2, 4, 6]] = 0.25
    np.testing.assert_allclose(P_y / P_y.sum(), expect, atol=10 * tol)
