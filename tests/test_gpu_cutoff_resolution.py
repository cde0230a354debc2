"""GPU: the discarded-weight cutoffs of the chi = 256 and chi = 512
configurations (eta = 1e-10 on 512-wide splits, eta = 1e-12 on 1024-wide
splits; truncation rule of Sec. II.B, Eq. 4) at full width, against the
oracle's FP64 split.

The FP32 split resolves the weight of a direction to about (eps32 sigma_F)^2,
so a cutoff decision is exact only up to the total weight that n directions
can carry at that level, delta = n (2 u)^2 W with u = 2^-24 the FP32 unit
roundoff.  The tests state that limit: the fidelity matches to 1e-5
relative at any width (the rank's boundary weight is far below it); the rank
must be exactly the oracle's where the boundary is resolvable (delta <<
eta W: the 512-wide eta = 1e-10 case), and otherwise lie within the delta band
of the rule's boundary (the 1024-wide eta = 1e-12 case, where delta > eta W:
the FP32 path does not resolve that cutoff)."""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import lib, random_unitary

pytestmark = pytest.mark.gpu
EPS32 = 2.0 ** -24


def _steep(n, decades):
    w = 10.0 ** (-decades * np.arange(n) / n)
    return np.sqrt(w / w.sum())


@pytest.mark.parametrize("nsites,chi,eta,decades,exact", [(18, 256, 1e-10, 11, True),
                                                          (20, 512, 1e-12, 11, False)])
def test_cutoff_at_full_width(nsites, chi, eta, decades, exact):
    P = lib()
    q0 = nsites // 2 - 1
    chis, sites, lams = synth.random_right_canonical(nsites, chi, seed=700 + chi, dtype=np.complex64)
    assert chis[q0] == chis[q0 + 2] == chi
    lams = [l.copy() for l in lams]
    lams[q0] = _steep(chi, decades)
    U = random_unitary(4, np.random.default_rng(chi))
    cfg = P.make_config(nsites, 2 * chi, eta, 2 + 2 * int(np.log2(2 * chi)), 0, 2, P.FP32)
    mps = P.MPS(cfg)
    mps.load(chis, sites, lams)
    f_gpu = float(mps.step([P.Cluster(q0, 2, 0, 0)], [U])[0])
    r_gpu = int(mps.bond_dims()[q0 + 1])
    A, B = sites[q0].astype(np.complex128), sites[q0 + 1].astype(np.complex128)
    th = np.einsum("st,atb->asb", U, np.tensordot(A, B, axes=([2], [0])).reshape(chi, 4, chi))
    (c,) = oracle.split_chain(th, lams[q0], 2 * chi, eta, floor=1e-6)
    n = 2 * chi
    s2 = c["s"] ** 2 / c["W"]
    tail = np.concatenate([np.cumsum(s2[::-1])[::-1], [0.0]])   # tail[r] = weight beyond the first r
    delta = n * (2 * EPS32) ** 2 * 1.0
    print(f"width {n} eta={eta:g}: r={r_gpu} (oracle {c['r']}) f={f_gpu:.12f} (oracle {c['f']:.12f}) "
          f"tail(r)={tail[r_gpu]:.3e} resolution delta={delta:.2e}")
    assert abs(f_gpu - c["f"]) <= 1e-5 * c["f"]
    assert abs(f_gpu - (1.0 - tail[r_gpu])) <= 1e-5
    if exact:
        assert delta < 0.1 * eta
        assert r_gpu == c["r"], (r_gpu, c["r"])
    else:
        assert delta > eta            # this width and cutoff are beyond the FP32 resolution
        lo, hi = sorted((r_gpu, c["r"]))
        # every rank between the two choices discards within delta of the cutoff
        assert tail[hi] <= eta + delta and tail[lo] <= eta + delta + np.sum(s2[lo:hi]), \
            (r_gpu, c["r"], tail[lo], tail[hi])
        assert abs(tail[r_gpu] - tail[c["r"]]) <= delta + eta, (tail[r_gpu], tail[c["r"]])
