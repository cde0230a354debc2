"""GPU: cluster-TEBD on the paper's random-structured circuits (Sec. IV.A slot
filling) with the full Clifford and non-Clifford gate sets of App. A (C-Y,
SWAP, sqrt(SWAP), C-H, C-S, C-T, P(3 pi/4), X^1/4, sqrt(W) ...), both control
orientations: exact runs against the state vector (FP64 to 1e-12, FP32 to
1e-5), and a truncated run against the oracle's run of the same circuit."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import as_oracle, download, fidelity_overlap, lib, run_gpu, statevector_of

pytestmark = pytest.mark.gpu


def _kinds(c):
    return set(int(k) for k in c.gates[:, 4])


@pytest.mark.parametrize("precision_name,tol", [("FP64", 1e-12), ("FP32", 1e-5)])
def test_exact_run_matches_statevector(precision_name, tol):
    P = lib()
    c = synth.paper_random_structured(12, 14, clifford=False, seed=11)
    assert {synth.CY, synth.CS, synth.CT, synth.SQSWAP, synth.SQW, synth.CH, synth.P} <= _kinds(c)
    mps, _ = run_gpu(c, 64, 0.0, 4 + 12, 0, 4, getattr(P, precision_name))
    ref = oracle.simulate(c, 64, 0.0, 4 + 12, 0, 4)
    assert list(mps.bond_dims()) == list(ref.chi())
    _, sites, _ = download(mps)
    psi = oracle.statevector(c)
    sv = statevector_of(sites)
    assert abs(np.vdot(psi, sv)) >= 1 - (1e-12 if precision_name == "FP64" else 1e-6)
    assert np.abs(sv - psi).max() < tol


def test_clifford_family_flat_spectra():
    P = lib()
    c = synth.paper_random_structured(14, 16, clifford=True, seed=12)
    assert {synth.CY, synth.SWAP, synth.Y} <= _kinds(c)
    mps, _ = run_gpu(c, 128, 0.0, 4 + 14, 0, 4, P.FP32)
    S = oracle.stabilizer_entropies(c)
    assert list(mps.bond_dims()) == [int(2 ** s) for s in S]
    for b in range(1, 14):
        lam = mps.lam(b)
        np.testing.assert_allclose(lam, np.full(len(lam), len(lam) ** -0.5), atol=2e-6)


@pytest.mark.parametrize("precision_name,rtol", [("FP64", 1e-10), ("FP32", 1e-5)])
def test_truncated_nonclifford_run_matches_oracle(precision_name, rtol):
    P = lib()
    c = synth.paper_random_structured(14, 40, clifford=False, seed=13)
    args = (16, 1e-4, 4 + 8, 0, 4)
    mps, log = run_gpu(c, *args, getattr(P, precision_name))
    ref = oracle.simulate(c, *args, floor=1e-13 if precision_name == "FP64" else 1e-6)
    assert list(mps.bond_dims()) == list(ref.chi())
    f_gpu = np.concatenate([f for (_, _, _, f) in log])
    np.testing.assert_allclose(f_gpu, ref.split_log()[:, 7], rtol=rtol)
    assert ref.logF < -1e-3                      # the run does truncate
    assert abs(mps.fidelity() / np.exp(ref.logF) - 1) <= 10 * rtol
    assert fidelity_overlap(ref, as_oracle(mps)) >= 1 - (1e-10 if precision_name == "FP64" else 1e-6)
