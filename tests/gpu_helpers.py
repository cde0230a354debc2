"""Shared helpers of the GPU parity tests (not collected as tests)."""
import numpy as np

import oracle
import synth


def lib():
    import paper_2502_19289_gb300 as P
    return P


def run_gpu(c, chi_max, cutoff, q_max, l_max, k_max, precision, stream=None):
    P = lib()
    circ = P.Circuit(c.n_qubits, c.gates, c.params)
    cfg = P.make_config(c.n_qubits, chi_max, cutoff, q_max, l_max, k_max, precision)
    log = []
    mps = P.simulate(circ, cfg, stream, callback=lambda s, e, cl, f: log.append(
        (s, e, [(x.q0, x.k) for x in cl], np.array(f))))
    return mps, log


def download(mps):
    chi = mps.bond_dims()
    sites = [mps.site(q) for q in range(mps.n)]
    lams = [mps.lam(b) for b in range(mps.n + 1)]
    return chi, sites, lams


def as_oracle(mps) -> oracle.MPS:
    _, sites, lams = download(mps)
    return oracle.MPS.from_arrays(sites, lams)


def fidelity_overlap(a: oracle.MPS, b: oracle.MPS) -> float:
    """|<a|b>| / (|a| |b|): after a truncation the right-canonical form is only
    approximately normalised (on both sides alike), so states are compared as rays."""
    return abs(a.overlap(b)) / np.sqrt(abs(a.overlap(a)) * abs(b.overlap(b)))


def statevector_of(sites):
    v = np.ones((1, 1), dtype=np.complex128)
    for s in sites:
        v = np.einsum("ia,asb->isb", v, s).reshape(-1, s.shape[2])
    return v.reshape(-1)


def oracle_split_rows(m: oracle.MPS):
    """Oracle split log as (q0, k, bond, m, n, r, f) rows (drop the step column)."""
    lg = m.split_log()
    return lg[:, 1:8]


def gpu_split_rows(log):
    return log


def random_unitary(d, rng):
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def contracted(sites, q0, k):
    t = sites[q0]
    for j in range(1, k):
        t = np.einsum("a...c,csb->a...sb", t, sites[q0 + j])
    return t.reshape(t.shape[0], -1, t.shape[-1])


def entangling_circuit(n, layers, seed):
    return synth.random_structured(n, layers, p1=1.0, p2=0.4,
                                   one_q={synth.H: 0.5, synth.T: 0.25, synth.X14: 0.25},
                                   two_q=(synth.CNOT, synth.CZ, synth.SQSWAP, synth.CH), seed=seed)
