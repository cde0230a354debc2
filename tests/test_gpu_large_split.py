"""GPU: one two-site cluster update at chi = 1024 on both sides (the split is a
2048 x 2048 problem) against the oracle's single-split fidelity.  Flat
(Porter-Thomas) and steep Schmidt spectra, with chi_max or the cutoff deciding
the rank.  The tolerance is 1e-5 relative on the split fidelity (Eq. 4)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib

pytestmark = pytest.mark.gpu
N, CHI, Q0 = 22, 1024, 10


def _haar(n, rng):
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


@pytest.fixture(scope="module")
def state():
    chis, sites, lams = synth.random_right_canonical(N, CHI, seed=2502, dtype=np.complex64)
    assert chis[Q0] == chis[Q0 + 1] == chis[Q0 + 2] == CHI
    return chis, sites, lams


def _steep(n):
    w = 10.0 ** (-12.0 * np.arange(n) / n)
    return np.sqrt(w / w.sum())


@pytest.mark.parametrize("spec,cutoff", [("flat", 1e-8), ("flat", 0.3), ("steep", 1e-10)])
def test_chi1024_split_matches_oracle(state, spec, cutoff):
    P = lib()
    chis, sites, lams = state
    lams = [l.copy() for l in lams]
    if spec == "steep":
        lams[Q0] = _steep(CHI)
    rng = np.random.default_rng(100 * (spec == "steep") + int(cutoff > 1e-3))
    U = _haar(4, rng)
    cfg = P.make_config(N, CHI, cutoff, 4 + 2 * 10, 0, 2, P.FP32)
    mps = P.MPS(cfg)
    mps.load(chis, sites, lams)
    f_gpu = float(mps.step([P.Cluster(Q0, 2, 0, 0)], [U])[0])
    r_gpu = int(mps.bond_dims()[Q0 + 1])
    lam_gpu = mps.lam(Q0 + 1)
    sweeps = tuple(int(x) for x in mps.split_log()[-1, 12:14])
    Bn = mps.site(Q0 + 1).reshape(r_gpu, -1).astype(np.complex128)
    orth = float(np.max(np.abs(Bn @ Bn.conj().T - np.eye(r_gpu))))

    A, B = sites[Q0].astype(np.complex128), sites[Q0 + 1].astype(np.complex128)
    th = np.tensordot(A, B, axes=([2], [0])).reshape(CHI, 4, CHI)
    th = np.einsum("st,atb->asb", U, th)
    M = th.reshape(2 * CHI, 2 * CHI)
    w = np.repeat(np.asarray(lams[Q0], dtype=np.float64), 2)
    r_ref, f_ref, W, s = oracle.split_fidelity(M, w, CHI, cutoff, floor=1e-6)
    cum = np.cumsum(s ** 2) / W
    print(f"{spec} cutoff={cutoff}: r={r_gpu} (oracle {r_ref}) f={f_gpu:.9f} (oracle {f_ref:.9f}) "
          f"sweeps pass1/pass2={sweeps} max|BB^H-I|={orth:.2e}")
    # the new site is right-isometric to FP32 accuracy (no drift of its row norms)
    assert orth <= 5e-5, orth

    # the kept subspace is optimal for the rank chosen: its weight equals the
    # top r_gpu values of the exact spectrum
    assert abs(f_gpu - cum[r_gpu - 1]) <= 1e-5 * cum[r_gpu - 1], (f_gpu, cum[r_gpu - 1], sweeps)
    # the rank follows the rule; a different choice only at a boundary within tolerance
    if r_gpu != r_ref:
        assert abs(cum[r_gpu - 1] - f_ref) <= 1e-5, (r_gpu, r_ref)
    assert abs(f_gpu - f_ref) <= 1e-5 * f_ref, (f_gpu, f_ref, r_gpu, r_ref)
    lam_ref = s[:r_gpu] / np.sqrt(np.sum(s[:r_gpu] ** 2))
    np.testing.assert_allclose(lam_gpu[:r_gpu], lam_ref, rtol=1e-3, atol=2e-6 * lam_ref[0])
