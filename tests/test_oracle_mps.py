"""Pins for the oracle's MPS cluster-TEBD (Sec. II.B-III.A) against the brute-force
state vector, closed forms (GHZ, product states), canonical-form invariants,
the stabilizer formalism (Clifford circuits), and Eq. 3 vs Eq. 5."""
import numpy as np
import pytest

import oracle
import synth

W1 = synth.WORKLOADS[1]


def _schmidt(psi, n, b):
    return np.linalg.svd(psi.reshape(1 << b, 1 << (n - b)), compute_uv=False)


@pytest.mark.parametrize("sample", range(4))
def test_cfg1_matches_statevector(sample):
    c = W1.circuit(sample, 1)
    psi = oracle.statevector(c)
    m = oracle.simulate(c, W1.chi_max, W1.cutoff, W1.q_max, 0, W1.k_max)
    sv = m.statevector()
    assert np.abs(sv - psi).max() <= 1e-12
    assert abs(np.vdot(psi, sv)) >= 1 - 1e-12
    assert abs(m.logF) < 1e-12            # nothing truncated: every f_j = 1


@pytest.mark.parametrize("seed", range(3))
def test_deeper_random_matches_statevector(seed):
    # n=10, 30 layers with long-range routing; several iterations and cluster sizes
    w = synth.reduced(2, 10, 30)
    c = w.circuit(seed, 2)
    psi = oracle.statevector(c)
    for q_max, k_max, l_max in ((12, 4, 0), (16, 6, 0), (20, 2, 1)):
        m = oracle.simulate(c, 1 << 10, 0.0, q_max, l_max, k_max)
        np.testing.assert_allclose(m.statevector(), psi, atol=1e-12)
        # canonical form: lambda_b are the Schmidt values of the state at bond b
        for b in range(1, 10):
            s = _schmidt(psi, 10, b)
            lam = m.lam(b)
            np.testing.assert_allclose(lam, s[:len(lam)], atol=1e-12)
            assert s[len(lam):].max(initial=0) < 1e-12


def test_sites_are_right_isometries():
    c = synth.reduced(2, 10, 20).circuit(7, 2)
    m = oracle.simulate(c, 16, 1e-6, 12, 0, 4)
    for q in range(10):
        B = m.site(q)
        Bm = B.reshape(B.shape[0], -1)
        np.testing.assert_allclose(Bm @ Bm.conj().T, np.eye(B.shape[0]), atol=1e-12)


def test_ghz_closed_form():
    n = 9
    c = synth.ghz_circuit(n)
    m = oracle.simulate(c, 64, 0.0, 8, 0, 4)
    assert list(m.chi()) == [1] + [2] * (n - 1) + [1]
    for b in range(1, n):
        np.testing.assert_allclose(m.lam(b), [2 ** -0.5, 2 ** -0.5], atol=1e-14)
    assert abs(m.amplitude([0] * n) - 2 ** -0.5) < 1e-14
    assert abs(m.amplitude([1] * n) - 2 ** -0.5) < 1e-14
    assert abs(m.amplitude([1] + [0] * (n - 1))) < 1e-14


def test_product_state_stays_chi_one():
    c = synth.product_circuit(7, seed=3)
    m = oracle.simulate(c, 64, 0.0, 8, 0, 4)
    assert list(m.chi()) == [1] * 8
    np.testing.assert_allclose(m.statevector(), oracle.statevector(c), atol=1e-14)


def test_clifford_tableau_and_flat_spectra():
    w = synth.reduced(3, 14, 20)
    c = w.circuit(1, 3)
    m = oracle.simulate(c, 1 << 8, 1e-12, 16, 0, 6)
    S = oracle.stabilizer_entropies(c)
    chi = m.chi()
    assert list(chi) == [2 ** s for s in S]                # Eq. 1 with equality
    for b in range(1, 14):
        np.testing.assert_allclose(m.lam(b), 2.0 ** (-S[b] / 2), atol=1e-12)
    psi = oracle.statevector(c)
    mag = np.abs(psi[np.abs(psi) > 1e-9])
    r = -2 * np.log2(mag[0])
    np.testing.assert_allclose(mag, 2.0 ** (-r / 2), atol=1e-12)   # uniform 2^{-r/2}
    assert abs(round(r) - r) < 1e-9 and len(mag) == 2 ** round(r)


def test_clifford_tableau_large_n():
    # n = 60 has no state vector; the tableau pins chi_b = 2^{S_b} directly
    c = synth.reduced(3, 60, 12).circuit(2, 3)
    m = oracle.simulate(c, 1 << 10, 1e-12, 24, 0, 8)
    S = oracle.stabilizer_entropies(c)
    assert list(m.chi()) == [2 ** s for s in S]
    assert abs(m.logF) < 1e-10


def test_stabilizer_entropy_against_statevector():
    for seed in range(4):
        c = synth.reduced(3, 10, 15).circuit(seed, 3)
        psi = oracle.statevector(c)
        S = oracle.stabilizer_entropies(c)
        for b in range(1, 10):
            s = _schmidt(psi, 10, b)
            assert int(np.sum(s > 1e-9)) == 2 ** S[b]


def test_truncated_norm_and_fidelity_eq3_vs_eq5():
    n = 12
    c = synth.random_structured(n, 24, p1=1.0, p2=0.4,
                                one_q={synth.H: 0.5, synth.T: 0.25, synth.X14: 0.25},
                                two_q=(synth.CNOT, synth.CZ, synth.SQSWAP, synth.CH), seed=0)
    exact = oracle.simulate(c, 1 << 12, 0.0, 14, 0, 4)
    trunc = oracle.simulate(c, 8, 1e-3, 10, 0, 4)
    assert trunc.logF < -1e-4                       # truncation actually happened
    F3 = abs(exact.overlap(trunc)) ** 2             # Eq. 3
    F5 = np.exp(trunc.logF)                         # Eq. 5
    # kept weight is renormalised; the Vidal form is only approximately
    # canonical after truncation, so the norm drifts by at most ~1 - F
    nrm = trunc.overlap(trunc).real
    assert abs(nrm - 1) < 2 * (1 - F5)
    assert abs(exact.overlap(exact) - 1) < 1e-12    # exact run: norm conserved
    assert F3 <= 1 + 1e-12
    assert abs(F3 - F5) < 0.25 * (1 - F5) + 1e-6    # "approximated accurately"


def test_standard_tebd_mode_matches():
    c = W1.circuit(2, 1)
    psi = oracle.statevector(c)
    m = oracle.simulate(c, 64, 0.0, 16, 1, 2)      # L_max = 1, k_max = 2: standard TEBD
    np.testing.assert_allclose(m.statevector(), psi, atol=1e-12)
    assert m.n_steps == oracle.asap_layers(12, c.gates)[1]


def test_amplitude_matches_statevector():
    c = W1.circuit(3, 1)
    psi = oracle.statevector(c)
    m = oracle.simulate(c, 64, 0.0, 16, 0, 4)
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = rng.integers(0, 2, 12)
        idx = int("".join(map(str, x)), 2)
        assert abs(m.amplitude(x) - psi[idx]) < 1e-13


@pytest.mark.parametrize("shape", [(7, 5), (5, 7), (16, 16), (40, 9), (3, 30)])
def test_jacobi_svd_against_library(shape):
    rng = np.random.default_rng(sum(shape))
    M = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    if shape == (16, 16):
        M[:, 8:] = M[:, :8] @ rng.standard_normal((8, 8))     # rank deficient
    s, Y = oracle.svd_right(M)
    ref = np.linalg.svd(M, compute_uv=False)
    np.testing.assert_allclose(s, ref, atol=1e-12 * ref[0])
    keep = s > 1e-10 * s[0]
    Yk = Y[:, keep]
    np.testing.assert_allclose(Yk.conj().T @ Yk, np.eye(keep.sum()), atol=1e-12)
    # M Y_k has orthogonal columns with norms s_k, and M = (M Y_k) Y_k^dagger
    MY = M @ Yk
    np.testing.assert_allclose(np.linalg.norm(MY, axis=0), s[keep], atol=1e-12 * s[0])
    np.testing.assert_allclose(MY @ Yk.conj().T, M, atol=1e-11 * s[0])


def test_truncation_rule_discarded_weight():
    # single k=2 cluster on a product state: the rule keeps the smallest r whose
    # discarded weight is <= cutoff * total (sorted descending), capped at chi_max.
    rng = np.random.default_rng(5)
    U = np.linalg.qr(rng.standard_normal((4, 4)) + 1j * rng.standard_normal((4, 4)))[0]
    m = oracle.MPS(2)
    f, r = m.cluster_update(0, 2, U, 4, 0.0)
    s_exact = np.linalg.svd(U[:, 0].reshape(2, 2), compute_uv=False)
    assert r[0] == 2 and abs(f[0] - 1) < 1e-14
    for cut, want in ((s_exact[1] ** 2 * 1.01, 1), (s_exact[1] ** 2 * 0.99, 2)):
        m = oracle.MPS(2)
        f, r = m.cluster_update(0, 2, U, 4, cut)
        assert r[0] == want
        if want == 1:
            np.testing.assert_allclose(f[0], s_exact[0] ** 2, atol=1e-14)
    m = oracle.MPS(2)
    f, r = m.cluster_update(0, 2, U, 1, 0.0)         # chi_max = 1
    assert r[0] == 1 and abs(f[0] - s_exact[0] ** 2) < 1e-14
    np.testing.assert_allclose(m.lam(1), [1.0])      # renormalised kept weight


def test_cluster_unitary_matches_kron():
    rng = np.random.default_rng(1)
    b = synth._Builder(6)
    b.g1(synth.H, 2)
    b.g2(synth.CNOT, 3, 2)          # control on the right: orientation matters
    b.g1(synth.T, 4)
    b.g2(synth.CZ, 3, 4)
    b.g2(synth.SQSWAP, 2, 3)
    c = b.build()
    layer, nl = oracle.asap_layers(6, c.gates)
    U = oracle.cluster_unitary(2, 3, c, layer, 0, nl)
    sub = synth.Circuit(3, c.gates.copy(), c.params)
    sub.gates[:, 1:3] = np.where(sub.gates[:, 1:3] >= 0, sub.gates[:, 1:3] - 2, -1)
    ref = np.stack([oracle.statevector(_with_prep(sub, x)) for x in range(8)], axis=1)
    np.testing.assert_allclose(U, ref, atol=1e-14)


def _with_prep(circ, x):
    """Prepend X gates so the circuit starts from basis state |x> (3 qubits)."""
    rows = [(1, q, -1, -1, synth.X) for q in range(3) if (x >> (2 - q)) & 1]
    g = np.concatenate([np.array(rows, np.int32).reshape(-1, 5), circ.gates])
    return synth.Circuit(3, g, np.concatenate([np.zeros(len(rows)), circ.params]))
