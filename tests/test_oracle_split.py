"""Pins of the oracle's single-split fidelity (Sec. II.C, Eqs. 4-5): closed-form
spectra with hand-derived ranks, and agreement with the oracle's own
cluster update (Jacobi SVD in C) on small random states."""
import numpy as np

import oracle
import synth


def _haar(n, rng):
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def _with_spectrum(s, m, n, w, rng):
    """M with diag(w) M = Q1 diag(s) Q2^H exactly (up to rounding)."""
    p = len(s)
    Q1 = _haar(m, rng)[:, :p]
    Q2 = _haar(n, rng)[:, :p]
    return (Q1 * s[None, :]) @ Q2.conj().T / np.asarray(w)[:, None]


def test_closed_form_ranks_and_fidelities():
    rng = np.random.default_rng(1)
    s2 = np.array([0.5, 0.3, 0.15, 0.05])
    s = np.sqrt(s2)
    w = rng.uniform(0.2, 2.0, size=6)            # non-uniform Schmidt weights on the rows
    M = _with_spectrum(s, 6, 5, w, rng)
    # (chi_max, cutoff, floor) -> (r, f) derived by hand from s^2
    cases = [((8, 0.0, 1e-13), (4, 1.0)),
             ((8, 0.06, 1e-13), (3, 0.95)),       # tail 0.05 <= 0.06 < 0.20
             ((8, 0.04, 1e-13), (4, 1.0)),        # tail 0.05 > 0.04
             ((8, 0.25, 1e-13), (2, 0.80)),       # 0.20 <= 0.25 < 0.50
             ((2, 0.0, 1e-13), (2, 0.80)),        # chi_max decides
             ((8, 0.0, 0.4), (3, 0.95)),          # s_3 = 0.224 < 0.4 * 0.707
             ((1, 0.0, 1e-13), (1, 0.50))]
    for (chi, eta, fl), (r_want, f_want) in cases:
        r, f, W, sv = oracle.split_fidelity(M, w, chi, eta, fl)
        np.testing.assert_allclose(sv[:4], s, atol=1e-12)
        assert abs(W - 1.0) < 1e-12
        assert r == r_want, (chi, eta, fl, r)
        assert abs(f - f_want) < 1e-12, (chi, eta, fl, f)


def _theta_matrix(sites, lams, q0, U):
    A, B = sites[q0], sites[q0 + 1]
    cl, cr = A.shape[0], B.shape[2]
    th = np.tensordot(A.astype(np.complex128), B.astype(np.complex128), axes=([2], [0]))
    th = th.reshape(cl, 4, cr)
    th = np.einsum("st,atb->asb", U, th)
    M = th.reshape(cl * 2, 2 * cr)
    w = np.repeat(np.asarray(lams[q0], dtype=np.float64), 2)
    return M, w


def test_matches_oracle_cluster_update():
    """Same theta through the C oracle's k=2 cluster update and through the
    single-split function: identical rank, fidelity to rounding."""
    rng = np.random.default_rng(7)
    for seed, chi_max, eta in [(3, 5, 0.0), (4, 64, 1e-2), (5, 7, 1e-3), (6, 64, 0.0)]:
        chis, sites, lams = synth.random_right_canonical(6, 8, seed)
        U = _haar(4, rng)
        q0 = 2
        M, w = _theta_matrix(sites, lams, q0, U)
        m = oracle.MPS.from_arrays(sites, lams)
        f_c, r_c = m.cluster_update(q0, 2, U, chi_max, eta)
        r, f, W, s = oracle.split_fidelity(M, w, chi_max, eta)
        assert int(r_c[0]) == r, (seed, r_c, r)
        assert abs(f_c[0] - f) < 1e-12, (seed, f_c, f)
        # the C oracle's Jacobi singular values agree with LAPACK's
        s_c, _ = oracle.svd_right(w[:, None] * M)
        np.testing.assert_allclose(s_c, s, rtol=1e-10, atol=1e-14)


def test_flat_spectrum_large_rank_budget():
    """A flat (Porter-Thomas) spectrum cut by chi_max at half its length: the
    kept weight equals the top half of s^2 (brute force over the sorted values)."""
    rng = np.random.default_rng(11)
    n = 64
    s = np.sort(np.sqrt(rng.exponential(1.0, n)))[::-1]
    s /= np.sqrt(np.sum(s ** 2))
    M = _with_spectrum(s, n, n, np.ones(n), rng)
    r, f, W, sv = oracle.split_fidelity(M, np.ones(n), n // 2, 1e-14)
    assert r == n // 2
    assert abs(f - np.sum(s[: n // 2] ** 2)) < 1e-12


def _cluster_theta(sites, q0, k, U):
    t = sites[q0].astype(np.complex128)
    for j in range(1, k):
        t = np.tensordot(t, sites[q0 + j].astype(np.complex128), axes=([t.ndim - 1], [0]))
    cl, cr = t.shape[0], t.shape[-1]
    return np.einsum("st,atb->asb", U, t.reshape(cl, 1 << k, cr))


def test_split_chain_matches_oracle_cluster_update():
    """The chained splits of a k = 3 and a k = 4 cluster against the C oracle's
    cluster update (its own Jacobi SVD, merge and remainder): same ranks at
    every bond, fidelities and spectra to rounding, truncated and untruncated."""
    rng = np.random.default_rng(21)
    for seed, k, chi, chi_max, eta in [(31, 3, 8, 64, 0.0), (32, 3, 8, 5, 1e-3),
                                       (33, 4, 4, 6, 1e-2), (34, 4, 8, 64, 1e-4)]:
        chis, sites, lams = synth.random_right_canonical(8, chi, seed)
        U = _haar(1 << k, rng)
        q0 = 2
        th = _cluster_theta(sites, q0, k, U)
        chain = oracle.split_chain(th, lams[q0], chi_max, eta)
        m = oracle.MPS.from_arrays(sites, lams)
        f_c, r_c = m.cluster_update(q0, k, U, chi_max, eta)
        assert [c["j"] for c in chain] == list(range(k - 1, 0, -1))
        assert [c["r"] for c in chain] == [int(x) for x in r_c], (seed, r_c)
        np.testing.assert_allclose([c["f"] for c in chain], f_c, rtol=1e-11)
        for c in chain:
            np.testing.assert_allclose(c["lam"], m.lam(q0 + c["j"]), rtol=1e-9, atol=1e-13)


def test_degenerate_cut_closed_form():
    """A stabilizer state has flat Schmidt spectra (Gottesman-Knill): six Bell
    pairs straddle the bond between qubits 6 and 7, and a Bell pair made on
    qubits 6, 7 by the cluster's H, CNOT gives a flat spectrum of 2^7 values.
    chi_max = 100 cuts inside that degenerate group: whichever 100 directions
    are kept, f = 100/128 (Eq. 4) and every kept lambda is 1/10."""
    c = synth.bell_pairs_circuit(14, [(j, j + 8) for j in range(6)])
    m = oracle.simulate(c, 64, 0.0, 16, 0, 4)
    assert list(m.chi()[6:9]) == [64, 64, 64]
    Hd = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    CN = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]])
    U = CN @ np.kron(Hd, np.eye(2))
    f, r = m.cluster_update(6, 2, U, 100, 0.0)
    assert int(r[0]) == 100 and m.chi()[7] == 100
    assert abs(f[0] - 100 / 128) < 1e-12
    np.testing.assert_allclose(m.lam(7), np.full(100, 0.1), atol=1e-12)
    # without the cut the same update is exact and the bond holds all 128 values
    m2 = oracle.simulate(c, 64, 0.0, 16, 0, 4)
    f2, r2 = m2.cluster_update(6, 2, U, 128, 0.0)
    assert int(r2[0]) == 128 and abs(f2[0] - 1.0) < 1e-12
    np.testing.assert_allclose(m2.lam(7), np.full(128, 2 ** -3.5), atol=1e-12)
