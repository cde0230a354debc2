"""GPU: the sketched split (randomized range finder, CholeskyQR2, Rayleigh-Ritz
on the projected problem, tail check) against the FP64 oracle's full SVD."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import as_oracle, contracted, fidelity_overlap, lib, random_unitary, run_gpu

pytestmark = pytest.mark.gpu


def _state(seed):
    # saturated profile up to chi 64 on 12 qubits: clusters near the left edge
    # have few rows and many columns, so their rank is far below the width
    return synth.random_right_canonical(12, 64, seed=seed)


def _run_cluster(P, q0, k, hints, cutoff, over, seed):
    chis, sites, lams = _state(seed)
    rng = np.random.default_rng(seed)
    U = random_unitary(1 << k, rng)
    cfg = P.make_config(12, 64, cutoff, 2 + 12 + 6, 0, 0, P.FP32, sketch_oversample=over,
                        power_iters=1, seed=99)
    m = P.MPS(cfg)
    m.load(chis, sites, lams)
    cl = P.Cluster(q0, k, 0, 1)
    for j, h in enumerate(hints):
        cl.rank_hint[j] = h
    f = m.step([cl], [U])
    ref = oracle.MPS.from_arrays(sites, lams)
    f_ref, r_ref = ref.cluster_update(q0, k, U, 64, cutoff)
    return m, ref, f, f_ref, m.split_log()


@pytest.mark.parametrize("q0,k", [(0, 3), (1, 3), (0, 4), (2, 2)])
def test_sketch_with_exact_rank_hint_matches_oracle(q0, k):
    P = lib()
    chis, _, _ = _state(5)
    bounds = [int(min(chis[q0] << j, (1 << (k - j)) * chis[q0 + k])) for j in range(1, k)]
    m, ref, f, f_ref, log = _run_cluster(P, q0, k, bounds, 1e-8, 4, seed=5)
    np.testing.assert_allclose(f, f_ref, rtol=1e-5)
    assert list(m.bond_dims()) == list(ref.chi())
    got = contracted([m.site(q) for q in range(12)], q0, k)
    want = contracted([ref.site(q) for q in range(12)], q0, k)
    np.testing.assert_allclose(got, want, atol=1e-5)
    attempted, fell_back = m.sketch_stats()
    assert attempted >= 1 and fell_back == 0
    assert log[:, 8].max() == 1            # at least one split was sketched
    for q in range(q0 + 1, q0 + k):
        B = m.site(q).reshape(m.bond_dims()[q], -1)
        np.testing.assert_allclose(B @ B.conj().T, np.eye(B.shape[0]), atol=1e-5)


def test_sketch_too_small_hint_falls_back():
    P = lib()
    q0, k = 1, 3
    m, ref, f, f_ref, log = _run_cluster(P, q0, k, [1, 1], 1e-8, 2, seed=6)
    attempted, fell_back = m.sketch_stats()
    assert attempted >= 1 and fell_back >= 1      # tail check rejected the sketch
    np.testing.assert_allclose(f, f_ref, rtol=1e-5)
    assert list(m.bond_dims()) == list(ref.chi())


def test_simulation_with_sketching_matches_oracle():
    """cfg2 statistics at n=20, 110 layers, Eq. 9 hints, sketch p=8."""
    P = lib()
    w = synth.reduced(2, 20, 110)
    c = w.circuit(0, 2)
    circ = P.Circuit(c.n_qubits, c.gates, c.params)
    cfg = P.make_config(20, 32, w.cutoff, w.q_max, 0, w.k_max, P.FP32, sketch_oversample=8)
    mps = P.MPS(cfg)
    start, n_sk = 0, 0
    while start < circ.n_layers:
        clusters, stop, f = P.run_iteration(mps, circ, start)
        if clusters:
            n_sk += int(mps.split_log()[:, 8].sum())
        start = stop
    ref = oracle.simulate(c, 32, w.cutoff, w.q_max, 0, w.k_max)
    assert n_sk > 0
    assert list(mps.bond_dims()) == list(ref.chi())
    assert fidelity_overlap(ref, as_oracle(mps)) >= 1 - 1e-6
    assert abs(mps.fidelity() / np.exp(ref.logF) - 1) <= 1e-5
