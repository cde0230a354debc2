"""split2_noalloc: the allocation-free two-site split, checked against the
regular apply_cluster + truncate_split entry points on two calls in a row.

Collected last on purpose (file name), so a failure here leaves every other
test already run."""
import numpy as np
import pytest

import synth
from gpu_helpers import lib, random_unitary

pytestmark = pytest.mark.gpu


def _case(P, torch, seed, chi, cutoff, n=4, q0=1, chi_max=None, steep=False):
    chis, sites, lams = synth.random_right_canonical(n, chi, seed=seed)
    chi_max = chi if chi_max is None else chi_max
    if steep:   # Schmidt weights spread over eight decades on the left bond
        w = 10.0 ** (-8.0 * np.arange(chis[q0]) / max(chis[q0] - 1, 1))
        lams = [l.copy() for l in lams]
        lams[q0] = np.sqrt(w / w.sum())
    rng = np.random.default_rng(seed)
    U = random_unitary(4, rng)
    cfg = P.make_config(n, chi_max, cutoff, 2 + 2 * int(np.ceil(np.log2(chi))) + 4, 0, 0, P.FP32)
    m = P.MPS(cfg)
    m.load(chis, sites, lams)
    # cluster tensor with the gate applied, no left weights (input of both paths)
    th = np.einsum("asc,ctb->astb", sites[q0].astype(np.complex64).astype(np.complex128),
                   sites[q0 + 1].astype(np.complex64).astype(np.complex128))
    cl, cr = th.shape[0], th.shape[-1]
    th = np.einsum("uv,avb->aub", U, th.reshape(cl, 4, cr))
    # regular entry points
    c = P.Cluster(q0, 2, 0, 1)
    m.apply_cluster(c, U)
    f_ref = m.truncate_split(c)
    r_ref = int(m.bond_dims()[q0 + 1])
    A_ref, B_ref = m.site(q0), m.site(q0 + 1)
    lam_ref = m.lam(q0 + 1)
    # allocation-free entry point; outputs sized exactly to the documented bound
    dev = torch.device("cuda")
    theta = torch.as_tensor(th.astype(np.complex64), device=dev).contiguous()
    lam_l = torch.as_tensor(lams[q0], dtype=torch.float64, device=dev)
    rmax = min(chi_max, 2 * cl, 2 * cr)
    A = torch.zeros(cl * 2 * rmax, dtype=torch.complex64, device=dev)
    B = torch.zeros(rmax * 2 * cr, dtype=torch.complex64, device=dev)
    lam = torch.zeros(rmax, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    r, f = P.split2_noalloc(theta.data_ptr(), lam_l.data_ptr(), cl, cr, chi_max, cutoff,
                            A.data_ptr(), B.data_ptr(), lam.data_ptr())
    assert 1 <= r <= rmax
    assert r == r_ref, (r, r_ref)
    np.testing.assert_allclose(f, f_ref[0], rtol=1e-5)
    np.testing.assert_allclose(lam.cpu().numpy()[:r], lam_ref, atol=1e-5)
    A = A.cpu().numpy()[: cl * 2 * r].reshape(cl, 2, r)
    B = B.cpu().numpy()[: r * 2 * cr].reshape(r, 2, cr)
    # the kept part of the cluster tensor, diag(lambda_l) A B: independent of the
    # basis chosen inside the kept space (rows of tiny Schmidt weight are resolved
    # only relative to the weighted norm, so the unweighted product is not
    # compared); directions at a chi_max cut inside a flat spectrum are resolved
    # to the split's 1e-5 weight tolerance, so the two paths agree to that level
    w = np.asarray(lams[q0], dtype=np.float64)[:, None, None, None]
    got = w * np.einsum("asm,mtb->astb", A, B)
    want = w * np.einsum("asm,mtb->astb", A_ref, B_ref)
    np.testing.assert_allclose(got, want, atol=2e-5 * float(np.max(np.abs(want))))
    Bm = B.reshape(r, -1)
    np.testing.assert_allclose(Bm @ Bm.conj().T, np.eye(r), atol=1e-5)
    return cl, cr, r


def test_noalloc_matches_regular_entry_points_twice():
    torch = pytest.importorskip("torch")
    P = lib()
    _case(P, torch, seed=11, chi=32, cutoff=1e-6)    # first call: sets up the scratch address
    _case(P, torch, seed=12, chi=64, cutoff=0.0)     # second call reuses the same scratch


def test_noalloc_full_size_bond_truncated_by_chi_max():
    """Both outer bonds at the 128 limit (a 256 x 256 split, eight Jacobi
    blocks), chi_max binding below the full rank, no cutoff."""
    torch = pytest.importorskip("torch")
    P = lib()
    cl, cr, r = _case(P, torch, seed=13, chi=128, cutoff=0.0, n=16, q0=7, chi_max=200)
    assert (cl, cr, r) == (128, 128, 200)


def test_noalloc_short_left_bond_with_steep_spectrum():
    """m = 2 chi_l < n = 2 chi_r and Schmidt weights over eight decades: the
    kept rank never exceeds the rank bound 2 chi_l of the split matrix."""
    torch = pytest.importorskip("torch")
    P = lib()
    cl, cr, r = _case(P, torch, seed=14, chi=64, cutoff=0.0, n=16, q0=4, steep=True)
    assert cl < cr and r <= 2 * cl, (cl, cr, r)


def test_noalloc_rejects_sizes_beyond_the_limit():
    pytest.importorskip("torch")
    P = lib()
    with pytest.raises(P.CtebdError, match="static scratch limit"):
        P.split2_noalloc(1, 1, 256, 8, 64, 0.0, 1, 1, 1)
