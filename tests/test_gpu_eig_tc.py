"""GPU: the Jacobi round update on the tensor cores (tcgen05, 3xTF32) against
the CUDA-core round update and the oracle's chained splits (Sec. III.A,
Fig. 2-3, Eq. 4).  Tensor cores forced on for every size (half-empty 128-row
tiles at 64 columns, odd pair counts, ragged row tiles), with chi_max and the
cutoff deciding ranks; the pass-2 refinement exercises the pair-flag paths
(identity rotations skipped, copy-only tiles)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib, random_unitary

pytestmark = pytest.mark.gpu


def _theta(sites, q0, k, U):
    t = sites[q0].astype(np.complex128)
    for j in range(1, k):
        t = np.tensordot(t, sites[q0 + j].astype(np.complex128), axes=([t.ndim - 1], [0]))
    cl, cr = t.shape[0], t.shape[-1]
    return np.einsum("st,atb->asb", U, t.reshape(cl, 1 << k, cr))


def _run(P, mode, n, chi, chi_max, cutoff, k, q0, sites, lams, chis, U):
    P.set_tensor_cores(mode)
    try:
        cfg = P.make_config(n, chi_max, cutoff, k + 2 * int(np.ceil(np.log2(max(chi_max, chi)))) + 2, 0, k, P.FP32)
        mps = P.MPS(cfg)
        mps.load(chis, sites, lams)
        f = np.asarray(mps.step([P.Cluster(q0, k, 0, 0)], [U]))
        return f, mps.bond_dims(), [mps.lam(q0 + j) for j in range(1, k)], mps.split_log(), mps
    finally:
        P.set_tensor_cores(1)


CASES = [  # n, chi (state), chi_max (>= chi: the loaded state must fit), cutoff, k, q0
    (8, 16, 16, 0.0, 2, 3),       # 32-wide splits: one pair, half-empty tiles
    (10, 32, 48, 1e-8, 2, 4),     # 64 wide, chi_max binding inside the width
    (12, 64, 64, 1e-3, 3, 4),     # odd pair counts (96-, 128-wide), cutoff binding
    (14, 128, 200, 1e-8, 2, 6),   # 256 wide
    (16, 160, 160, 1e-6, 2, 7),   # 320 wide: ragged 128-row V tiles
    (20, 512, 800, 1e-8, 2, 9),   # 1024 wide
]


@pytest.mark.parametrize("n,chi,chi_max,cutoff,k,q0", CASES)
def test_tensor_core_round_update_matches(n, chi, chi_max, cutoff, k, q0):
    P = lib()
    chis = synth.bond_dims_saturated(n, chi)
    chis, sites, lams = synth.random_right_canonical(n, chi, seed=900 + chi, dtype=np.complex64, chis=chis)
    U = random_unitary(1 << k, np.random.default_rng(chi + k))
    f_tc, chi_tc, lam_tc, log_tc, m_tc = _run(P, 2, n, chi, chi_max, cutoff, k, q0, sites, lams, chis, U)
    f_sm, chi_sm, lam_sm, log_sm, _ = _run(P, 0, n, chi, chi_max, cutoff, k, q0, sites, lams, chis, U)
    ref = oracle.split_chain(_theta(sites, q0, k, U), lams[q0], chi_max, cutoff, floor=1e-6)
    print(f"n={n} chi={chi} k={k}: f tc {f_tc} simt {f_sm} oracle {[c['f'] for c in ref]}; "
          f"sweeps tc {log_tc[:, 12:14].tolist()} simt {log_sm[:, 12:14].tolist()}")
    for i, c in enumerate(ref):
        bond = q0 + c["j"]
        s2 = c["s"] ** 2
        cum = np.cumsum(s2) / np.sum(s2)
        for f, chi_out, lam in ((f_tc, chi_tc, lam_tc), (f_sm, chi_sm, lam_sm)):
            r = int(chi_out[bond])
            assert abs(f[i] - c["f"]) <= 1e-5 * c["f"], (bond, f[i], c["f"])
            if r != c["r"]:
                assert abs(cum[r - 1] - c["f"]) <= 1e-5, (bond, r, c["r"])
            else:
                np.testing.assert_allclose(lam[c["j"] - 1][:r], c["lam"][:r], rtol=1e-3,
                                           atol=2e-6 * c["lam"][0])
    # the new sites stay isometric through the tensor-core rotations
    for j in range(1, k):
        B = m_tc.site(q0 + j).reshape(int(chi_tc[q0 + j]), -1).astype(np.complex128)
        assert np.max(np.abs(B @ B.conj().T - np.eye(B.shape[0]))) <= 5e-5


def test_tensor_core_round_update_through_a_run():
    """A whole entangling run (growing bonds, several clusters per iteration,
    many sweep shapes) with every round update on the tensor cores, against the
    oracle's run of the same circuit: bond dimensions, every split's fidelity
    and the state."""
    P = lib()
    from gpu_helpers import as_oracle, entangling_circuit, fidelity_overlap, run_gpu
    c = entangling_circuit(14, 24, seed=31)
    args = (48, 1e-7, 4 + 12, 0, 4)
    P.set_tensor_cores(2)
    try:
        mps, log = run_gpu(c, *args, P.FP32)
    finally:
        P.set_tensor_cores(1)
    ref = oracle.simulate(c, *args, floor=1e-6)
    assert list(mps.bond_dims()) == list(ref.chi())
    f_gpu = np.concatenate([f for (_, _, _, f) in log])
    np.testing.assert_allclose(f_gpu, ref.split_log()[:, 7], rtol=1e-5)
    assert abs(mps.fidelity() / np.exp(ref.logF) - 1) <= 1e-5
    assert fidelity_overlap(ref, as_oracle(mps)) >= 1 - 1e-6
