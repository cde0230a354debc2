"""GPU: truncation inside a degenerate (flat) Schmidt spectrum, the case in
which several kept subspaces are equally optimal (truncation rule of
Sec. II.B, fidelity of Eq. 4).  Only what is unique is compared: the rank, the
split fidelity, the kept spectrum and the fidelity product.

The input is a stabilizer state with flat spectra (six Bell pairs straddling
the middle bond of 14 qubits, qubits 6 and 7 free); the cluster on qubits 6, 7
makes a seventh Bell pair across bond 7, so its split sees 128 equal Schmidt
values and chi_max = 100 cuts inside them: f = 100/128 and lambda = 1/10
whichever 100 directions are kept.  The oracle reaches the same closed form."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import download, lib

pytestmark = pytest.mark.gpu


def _state():
    c = synth.bell_pairs_circuit(14, [(j, j + 8) for j in range(6)])
    return oracle.simulate(c, 64, 0.0, 16, 0, 4)


def _bell_gate():
    Hd = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    CN = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]])
    return (CN @ np.kron(Hd, np.eye(2))).astype(np.complex128)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("chi_max", [100, 127, 65])
def test_cut_inside_flat_spectrum(prec, chi_max):
    P = lib()
    ref = _state()
    chis = ref.chi()
    sites = [ref.site(q) for q in range(14)]
    lams = [ref.lam(b) for b in range(15)]
    cfg = P.make_config(14, chi_max, 0.0, 2 + 2 * 7 + 2, 0, 4, P.FP32 if prec == "fp32" else P.FP64)
    mps = P.MPS(cfg)
    mps.load(chis, sites, lams)
    U = _bell_gate()
    # a second, untruncated cluster in the same step: a CZ inside the paired block
    CZ = np.diag([1, 1, 1, -1]).astype(np.complex128)
    f = mps.step([P.Cluster(2, 2, 0, 1), P.Cluster(6, 2, 0, 1)], [CZ, U])
    tol_f = 1e-6 if prec == "fp32" else 1e-12
    tol_l = 1e-5 if prec == "fp32" else 1e-12
    chi = mps.bond_dims()
    assert chi[7] == chi_max
    assert abs(f[0] - 1.0) < tol_f                       # the CZ cluster keeps everything
    assert abs(f[1] - chi_max / 128) < tol_f * chi_max / 128, (f, chi_max / 128)
    np.testing.assert_allclose(mps.lam(7), np.full(chi_max, chi_max ** -0.5), atol=tol_l)
    assert abs(mps.fidelity() - chi_max / 128) < tol_f
    # the oracle takes the same decision and reaches the same closed form
    ref.cluster_update(2, 2, CZ, chi_max, 0.0)
    fo, ro = ref.cluster_update(6, 2, U, chi_max, 0.0)
    assert list(ref.chi()) == list(chi)
    assert abs(fo[0] - f[1]) < tol_f
    # the new right site is an isometry whichever subspace was kept
    B = mps.site(7).reshape(chi_max, -1)
    np.testing.assert_allclose(B @ B.conj().T, np.eye(chi_max), atol=10 * tol_l)
    # bonds away from the cut keep their flat spectra exactly
    _, _, lam_after = download(mps)
    for b in (3, 6, 8):
        np.testing.assert_allclose(lam_after[b], np.full(len(lam_after[b]), len(lam_after[b]) ** -0.5),
                                   atol=tol_l)
