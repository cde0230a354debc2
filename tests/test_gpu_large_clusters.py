"""GPU: cluster updates of k = 3 and k = 4 qubits at chi >= 512 on both outer
bonds, compared split by split with the oracle's chained truncated splits
(Sec. III.A, Fig. 2 and Fig. 3; truncation rule of Sec. II.B; Eq. 4): the
k - 1 splits run right to left, every one compared on its fidelity (1e-5
relative), its rank and its kept spectrum.  Flat (Porter-Thomas) spectra with
chi_max deciding the rank, and a steep left spectrum with the cutoff deciding
it.  The merge chain (k - 1 products), the cluster unitary on 2^k = 8 and 16
and multi-level splits at these sizes are all on the path."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib, random_unitary

pytestmark = pytest.mark.gpu


def _steep(n, decades):
    w = 10.0 ** (-decades * np.arange(n) / n)
    return np.sqrt(w / w.sum())


def _theta(sites, q0, k, U):
    t = sites[q0].astype(np.complex128)
    for j in range(1, k):
        t = np.tensordot(t, sites[q0 + j].astype(np.complex128), axes=([t.ndim - 1], [0]))
    cl, cr = t.shape[0], t.shape[-1]
    return np.einsum("st,atb->asb", U, t.reshape(cl, 1 << k, cr))


CASES = [  # (n sites, chi, k, q0, left spectrum, cutoff)
    (22, 512, 3, 9, "flat", 1e-8),
    (22, 512, 4, 9, "flat", 1e-8),
    (22, 512, 4, 9, "steep", 1e-10),
    (24, 1024, 3, 10, "flat", 1e-8),
]


@pytest.mark.parametrize("n,chi,k,q0,spec,cutoff", CASES)
def test_cluster_splits_match_oracle(n, chi, k, q0, spec, cutoff):
    P = lib()
    chis, sites, lams = synth.random_right_canonical(n, chi, seed=600 + k + chi, dtype=np.complex64)
    assert chis[q0] == chis[q0 + k] == chi
    lams = [l.copy() for l in lams]
    if spec == "steep":
        lams[q0] = _steep(chi, 10)
    rng = np.random.default_rng(k * 1000 + chi)
    U = random_unitary(1 << k, rng)
    cfg = P.make_config(n, chi, cutoff, k + 2 * int(np.log2(chi)), 0, k, P.FP32)
    mps = P.MPS(cfg)
    mps.load(chis, sites, lams)
    f_gpu = np.asarray(mps.step([P.Cluster(q0, k, 0, 0)], [U]))
    chi_gpu = mps.bond_dims()
    log = mps.split_log()
    ref = oracle.split_chain(_theta(sites, q0, k, U), lams[q0], chi, cutoff, floor=1e-6)
    assert len(f_gpu) == len(ref) == k - 1
    for i, c in enumerate(ref):
        bond = q0 + c["j"]
        r_gpu, r_ref = int(chi_gpu[bond]), c["r"]
        row = log[i]
        assert int(row[2]) == bond and int(row[3]) == c["m"], (row[:6], c["m"])
        s2 = c["s"] ** 2
        cum = np.cumsum(s2) / np.sum(s2)
        print(f"k={k} chi={chi} {spec} bond {bond}: r={r_gpu} (oracle {r_ref}) "
              f"f={f_gpu[i]:.9f} (oracle {c['f']:.9f}) sweeps={tuple(int(x) for x in row[12:14])}")
        assert abs(f_gpu[i] - c["f"]) <= 1e-5 * c["f"], (bond, f_gpu[i], c["f"])
        if r_gpu != r_ref:   # a different rank only where the rule's boundary is within tolerance
            assert abs(cum[r_gpu - 1] - c["f"]) <= 1e-5, (bond, r_gpu, r_ref)
        r = min(r_gpu, r_ref)
        lam = mps.lam(bond)
        np.testing.assert_allclose(lam[:r], c["lam"][:r] * np.sqrt(c["f"] / cum[r_gpu - 1]) if r_gpu != r_ref
                                   else c["lam"][:r], rtol=1e-3, atol=2e-6 * c["lam"][0])
        B = mps.site(bond).reshape(r_gpu, -1).astype(np.complex128)
        assert np.max(np.abs(B @ B.conj().T - np.eye(r_gpu))) <= 5e-5
    assert abs(mps.fidelity() - np.prod([c["f"] for c in ref])) <= 1e-5 * np.prod([c["f"] for c in ref])
