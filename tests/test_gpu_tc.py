"""GPU: the tcgen05 tile engine (3xTF32 complex products on packed operands)
against a complex128 reference product, at tile multiples and ragged sizes."""
import numpy as np
import pytest

from gpu_helpers import lib

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,K,N", [(128, 32, 64), (256, 96, 128), (384, 64, 192), (256, 2048, 128),
                                   (200, 37, 50), (1000, 301, 130), (1, 5, 3), (129, 16, 65)])
def test_tc_cgemm_matches_reference(M, K, N):
    torch = pytest.importorskip("torch")
    P = lib()
    rng = np.random.default_rng(M + K + N)
    A = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))).astype(np.complex64)
    B = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))).astype(np.complex64)
    dev = torch.device("cuda")
    Ad, Bd = torch.as_tensor(A, device=dev), torch.as_tensor(B, device=dev)
    Cd = torch.zeros((M, N), dtype=torch.complex64, device=dev)
    torch.cuda.synchronize()
    P.tc_cgemm(Ad.data_ptr(), Bd.data_ptr(), Cd.data_ptr(), M, K, N)
    C = Cd.cpu().numpy()
    ref = A.astype(np.complex128) @ B.astype(np.complex128)
    err = np.abs(C - ref).max() / np.abs(ref).max()
    assert err < 2e-6, err          # FP32-level at any K (1xTF32 would be ~1e-3)


@pytest.fixture
def tensor_cores_forced():
    P = lib()
    P.set_tensor_cores(2)
    yield
    P.set_tensor_cores(1)


def test_cluster_updates_with_tensor_core_gemms_match_oracle(tensor_cores_forced):
    """Every FP32 GEMM of the update on the tensor cores (merge, U, Gram,
    projections): same parity targets as the CUDA-core path."""
    import oracle
    import synth
    from gpu_helpers import as_oracle, fidelity_overlap, run_gpu
    P = lib()
    w = synth.reduced(2, 20, 110)
    c = w.circuit(0, 2)
    for chi in (256, 32):
        args = (chi, w.cutoff, w.q_max, 0, w.k_max)
        mps, log = run_gpu(c, *args, P.FP32)
        ref = oracle.simulate(c, *args)
        assert list(mps.bond_dims()) == list(ref.chi())
        assert fidelity_overlap(ref, as_oracle(mps)) >= 1 - 1e-6
        f_gpu = np.concatenate([f for (_, _, _, f) in log])
        np.testing.assert_allclose(f_gpu, ref.split_log()[:, 7], rtol=1e-5)
