"""GPU: closed forms and degenerate cases.  GHZ states have a degenerate
Schmidt spectrum (two equal values per bond); product states keep every bond
at dimension 1; a step with no clusters leaves the state and F unchanged."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import download, lib, run_gpu, statevector_of

pytestmark = pytest.mark.gpu
TOL = {"FP64": 1e-12, "FP32": 2e-6}


@pytest.mark.parametrize("precision_name", ["FP64", "FP32"])
def test_ghz_closed_form(precision_name):
    P = lib()
    n = 12
    c = synth.ghz_circuit(n)
    mps, _ = run_gpu(c, 4, 0.0, 8, 0, 4, getattr(P, precision_name))
    tol = TOL[precision_name]
    assert list(mps.bond_dims()) == [1] + [2] * (n - 1) + [1]
    for b in range(1, n):
        np.testing.assert_allclose(mps.lam(b), [2 ** -0.5, 2 ** -0.5], atol=tol)
    assert abs(mps.amplitude(np.zeros(n, np.uint8)) - 2 ** -0.5) < tol
    assert abs(mps.amplitude(np.ones(n, np.uint8)) - 2 ** -0.5) < tol
    one_hot = np.zeros(n, np.uint8)
    one_hot[0] = 1
    assert abs(mps.amplitude(one_hot)) < tol
    assert abs(mps.fidelity() - 1.0) < tol


@pytest.mark.parametrize("precision_name", ["FP64", "FP32"])
def test_product_state_stays_chi_one(precision_name):
    P = lib()
    c = synth.product_circuit(9, seed=3)
    mps, _ = run_gpu(c, 4, 0.0, 8, 0, 4, getattr(P, precision_name))
    assert list(mps.bond_dims()) == [1] * 10
    _, sites, _ = download(mps)
    np.testing.assert_allclose(statevector_of(sites), oracle.statevector(c), atol=TOL[precision_name])


def test_empty_step_changes_nothing():
    P = lib()
    c = synth.ghz_circuit(6)
    mps, _ = run_gpu(c, 4, 0.0, 8, 0, 4, P.FP32)
    before = statevector_of(download(mps)[1])
    f = mps.step([], [])
    assert len(f) == 0
    np.testing.assert_array_equal(statevector_of(download(mps)[1]), before)
    assert abs(mps.fidelity() - 1.0) < 1e-6


@pytest.mark.parametrize("graphs", [True, False])
def test_sweep_cap_reports_numeric_error(graphs):
    """A Jacobi eigen-solve still rotating at the sweep cap is an error
    (CTEBD_ERR_NUMERIC), never a silently unconverged split.  One sweep cannot
    diagonalise a random 128-wide split; the default cap solves it."""
    P = lib()
    chis, sites, lams = synth.random_right_canonical(12, 64, seed=77)
    U = np.linalg.qr(np.random.default_rng(77).standard_normal((4, 4)))[0].astype(np.complex128)
    cfg = P.make_config(12, 64, 1e-8, 2 + 12 + 2, 0, 2, P.FP32)
    cap = P.max_sweeps()
    try:
        P.set_sweep_graphs(2 if graphs else 0)
        P.set_max_sweeps(1)
        mps = P.MPS(cfg)
        mps.load(chis, sites, lams)
        with pytest.raises(P.CtebdError, match="still rotating after 1 sweeps"):
            mps.step([P.Cluster(5, 2, 0, 0)], [U])
    finally:
        P.set_max_sweeps(cap)
        P.set_sweep_graphs(1)
    mps = P.MPS(cfg)
    mps.load(chis, sites, lams)
    f = mps.step([P.Cluster(5, 2, 0, 0)], [U])
    assert 0.0 < f[0] <= 1.0
    with pytest.raises(P.CtebdError):
        P.set_max_sweeps(0)
