"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only *generates inputs*: gate lists of random-structured circuits
(Sec. IV.A of the paper, with the per-workload probabilities fixed below) and
random MPS states in right-canonical (Vidal) form.  It holds none of the
method's arithmetic: no layering, no partitioning, no contraction, no SVD.

Gate records
------------
A circuit is a time-ordered list of gates.  Each gate is a row
``(n_q, q0, q1, q2, kind)`` of an int32 array plus one float64 parameter.
Qubits are 0-indexed; for a two-qubit gate ``q0`` is the first listed qubit
(the control of a controlled gate, i.e. the most significant bit of the 4x4
gate matrix, App. A) and ``q1`` the second.  Unused slots hold -1.

The integer gate codes below are an interface shared by every consumer; the
matrices they name are the ones printed in App. A (plus S = P(pi/2)).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# ---- gate codes (App. A; S = P(pi/2) from the phase-gate definition) -------
H, X, Y, Z, S, T, P, X14, SQW = 1, 2, 3, 4, 5, 6, 7, 8, 9
CNOT, CY, CZ, SWAP, CH, CS, CT, SQSWAP, CP = 10, 11, 12, 13, 14, 15, 16, 17, 18
ONE_QUBIT = (H, X, Y, Z, S, T, P, X14, SQW)
TWO_QUBIT = (CNOT, CY, CZ, SWAP, CH, CS, CT, SQSWAP, CP)
CLIFFORD = (H, X, Y, Z, S, CNOT, CY, CZ, SWAP)
NAMES = {H: "H", X: "X", Y: "Y", Z: "Z", S: "S", T: "T", P: "P", X14: "X^1/4",
         SQW: "sqrtW", CNOT: "CNOT", CY: "CY", CZ: "CZ", SWAP: "SWAP", CH: "CH",
         CS: "CS", CT: "CT", SQSWAP: "sqrtSWAP", CP: "CP"}


@dataclass
class Circuit:
    n_qubits: int
    gates: np.ndarray          # int32 (n_gates, 5): n_q, q0, q1, q2, kind
    params: np.ndarray         # float64 (n_gates,)

    @property
    def n_gates(self) -> int:
        return int(self.gates.shape[0])


class _Builder:
    def __init__(self, n):
        self.n = n
        self.rows: list[tuple[int, int, int, int, int]] = []
        self.params: list[float] = []

    def g1(self, kind, q, param=0.0):
        self.rows.append((1, q, -1, -1, kind))
        self.params.append(param)

    def g2(self, kind, a, b, param=0.0):
        self.rows.append((2, a, b, -1, kind))
        self.params.append(param)

    def build(self) -> Circuit:
        g = np.array(self.rows, dtype=np.int32).reshape(-1, 5)
        return Circuit(self.n, g, np.array(self.params, dtype=np.float64))


def random_structured(n: int, n_layers: int, *, p1: float, p2: float,
                      one_q: dict[int, float], two_q: tuple[int, ...],
                      long_range_frac: float = 0.0, long_range_dmax: int = 4,
                      seed: int = 0) -> Circuit:
    """Random-structured circuit (Sec. IV.A), generated layer by layer.

    In every generation layer the nearest-neighbour bonds are scanned left to
    right; a two-qubit gate (uniform over ``two_q``, control on the lower
    qubit) is put on bond (i, i+1) with probability ``p2`` when both qubits
    are still free.  With probability ``long_range_frac`` such a gate instead
    couples (i, i+d), d uniform in {2..long_range_dmax}; it is emitted routed
    by a SWAP chain that brings qubit i+d next to i, the gate on (i, i+1),
    and the reversed chain (Sec. IV.A, routing of long-range gates).  Every
    qubit left free then gets a one-qubit gate with probability ``p1`` drawn
    from the distribution ``one_q``.  The emitted list is time-ordered; layer
    numbers are assigned later by whoever consumes it.
    """
    rng = np.random.default_rng(seed)
    kinds1 = np.array(list(one_q.keys()), dtype=np.int64)
    probs1 = np.array(list(one_q.values()), dtype=np.float64)
    probs1 = probs1 / probs1.sum()
    b = _Builder(n)
    for _ in range(n_layers):
        free = np.ones(n, dtype=bool)
        i = 0
        while i < n - 1:
            if free[i] and free[i + 1] and rng.random() < p2:
                kind = int(two_q[rng.integers(len(two_q))])
                d = 1
                if long_range_frac > 0.0 and rng.random() < long_range_frac:
                    d = int(rng.integers(2, long_range_dmax + 1))
                    if i + d >= n or not free[i:i + d + 1].all():
                        d = 1
                if d == 1:
                    b.g2(kind, i, i + 1)
                    free[i] = free[i + 1] = False
                    i += 2
                    continue
                chain = [(j - 1, j) for j in range(i + d, i + 1, -1)]
                for a, c in chain:
                    b.g2(SWAP, a, c)
                b.g2(kind, i, i + 1)
                for a, c in reversed(chain):
                    b.g2(SWAP, a, c)
                free[i:i + d + 1] = False
                i += d + 1
                continue
            i += 1
        for q in range(n):
            if free[q] and rng.random() < p1:
                b.g1(int(kinds1[rng.choice(len(kinds1), p=probs1)]), q)
    return b.build()


# the gate sets of the two random-structured circuit families (Sec. IV.A):
# Clifford, and the same sets extended by non-Clifford gates (one in two of
# each set non-Clifford); P(3 pi / 4) carries its angle as the parameter
PAPER_CLIFFORD_1Q = ((H, 0.0), (X, 0.0), (Y, 0.0), (Z, 0.0))
PAPER_CLIFFORD_2Q = (CNOT, CY, CZ, SWAP)
PAPER_NONCLIFFORD_1Q = PAPER_CLIFFORD_1Q + ((T, 0.0), (P, 0.75 * math.pi), (X14, 0.0), (SQW, 0.0))
PAPER_NONCLIFFORD_2Q = PAPER_CLIFFORD_2Q + (CH, CS, CT, SQSWAP)


def paper_random_structured(n: int, n_layers: int, *, clifford: bool, seed: int = 0,
                            p_two: float = 0.5) -> Circuit:
    """Random-structured circuit as the paper generates it (Sec. IV.A): every
    slot of every layer is filled, left to right, with a random one-qubit gate
    or -- with probability p_two = 0.5, when a right neighbour is still free in
    the layer -- a random two-qubit gate on the slot and its right neighbour,
    until all layers are complete.  Gates are drawn uniformly from the
    Clifford sets {H, X, Y, Z} and {CNOT, C-Y, C-Z, SWAP}, or from those sets
    extended by {T, P(3 pi/4), X^1/4, sqrt(W)} and {C-H, C-S, C-T, sqrt(SWAP)}
    (clifford=False).  The control of an asymmetric two-qubit gate is either
    qubit, uniformly (first listed = control)."""
    rng = np.random.default_rng(seed)
    one = PAPER_CLIFFORD_1Q if clifford else PAPER_NONCLIFFORD_1Q
    two = PAPER_CLIFFORD_2Q if clifford else PAPER_NONCLIFFORD_2Q
    b = _Builder(n)
    for _ in range(n_layers):
        q = 0
        while q < n:
            if q + 1 < n and rng.random() < p_two:
                kind = int(two[rng.integers(len(two))])
                if rng.random() < 0.5:
                    b.g2(kind, q, q + 1)
                else:
                    b.g2(kind, q + 1, q)
                q += 2
            else:
                kind, param = one[rng.integers(len(one))]
                b.g1(int(kind), q, float(param))
                q += 1
    return b.build()


# ---- workload definitions (seed = 1000 * config + sample) -------------------
@dataclass
class Workload:
    name: str
    n_qubits: int
    n_layers: int
    chi_max: int
    cutoff: float
    k_max: int
    precision: str              # "fp64" | "fp32"
    p1: float
    p2: float
    one_q: dict = field(default_factory=dict)
    two_q: tuple = (CNOT, CZ)
    long_range_frac: float = 0.0

    @property
    def q_max(self) -> int:
        # Eq. 7 memory bound chosen so that any k <= k_max cluster between two
        # chi_max bonds fits: Q_max = k_max + 2 log2 chi_max.
        return self.k_max + 2 * int(math.log2(self.chi_max))

    def circuit(self, sample: int = 0, config_id: int = 0) -> Circuit:
        return random_structured(
            self.n_qubits, self.n_layers, p1=self.p1, p2=self.p2,
            one_q=self.one_q, two_q=self.two_q,
            long_range_frac=self.long_range_frac, seed=1000 * config_id + sample)


WORKLOADS = {
    # n=12, 10 layers, H/S/T with p=0.5, CNOT/CZ with p=0.3, exact (chi 64).
    1: Workload("cfg1-exact-n12", 12, 10, 64, 0.0, 4, "fp64", 0.5, 0.3,
                {H: 1 / 3, S: 1 / 3, T: 1 / 3}),
    # n=100, 50 layers, Clifford+T (10% T), 10% long-range pairs, chi 256.
    2: Workload("cfg2-n100-chi256", 100, 50, 256, 1e-10, 6, "fp32", 0.5, 0.3,
                {T: 0.10, H: 0.45, S: 0.45}, long_range_frac=0.10),
    # n=1000, 100 layers, Clifford only (H, S, CNOT, CZ), p2=0.25, chi 512.
    3: Workload("cfg3-n1000-clifford-chi512", 1000, 100, 512, 1e-12, 8, "fp32",
                0.5, 0.25, {H: 0.5, S: 0.5}),
    # n=500, 100 layers, Clifford+T (20% T), chi 1024, cutoff 1e-8, k_max 4.
    4: Workload("cfg4-n500-chi1024", 500, 100, 1024, 1e-8, 4, "fp32", 0.5, 0.3,
                {T: 0.20, H: 0.40, S: 0.40}),
}


def cfg5_circuits(n_circuits: int = 64, seed: int = 5000):
    """64 independent circuits: n ~ U[50,300], layers ~ U[40,100], T ~ U[5%,25%]."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n_circuits):
        n = int(rng.integers(50, 301))
        L = int(rng.integers(40, 101))
        t = float(rng.uniform(0.05, 0.25))
        out.append(random_structured(n, L, p1=0.5, p2=0.3,
                                     one_q={T: t, H: (1 - t) / 2, S: (1 - t) / 2},
                                     two_q=(CNOT, CZ), seed=seed + 1 + c))
    return out


def reduced(config_id: int, n_qubits: int, n_layers: int) -> Workload:
    """Same gate statistics as a workload, at a size the oracle finishes."""
    w = WORKLOADS[config_id]
    return Workload(w.name + f"-reduced-n{n_qubits}-L{n_layers}", n_qubits, n_layers,
                    w.chi_max, w.cutoff, w.k_max, w.precision, w.p1, w.p2,
                    dict(w.one_q), w.two_q, w.long_range_frac)


def fig7_circuit() -> Circuit:
    """The entangling gates named in the caption of Fig. 7 (8 qubits).

    Layers 1-2 pair (1,2),(3,4),(5,6),(7,8); layer 3 has U_(6,7); layer 4 has
    U_(1,2) and U_(5,6); layer 5 has U_(4,5) (1-indexed in the paper).  The
    figure image is not available: one-qubit H gates on qubits 1-4 at layer 3
    are added so that earliest-layer placement (Sec. II.A) puts U_(1,2) at
    layer 4 as the caption states (0-indexed qubits here).
    """
    b = _Builder(8)
    for _ in range(2):
        for i in (0, 2, 4, 6):
            b.g2(CNOT, i, i + 1)
    b.g2(CZ, 5, 6)
    for q in (0, 1, 2, 3):
        b.g1(H, q)
    b.g2(CNOT, 0, 1)
    b.g2(CNOT, 4, 5)
    b.g2(CZ, 3, 4)
    return b.build()


def ghz_circuit(n: int) -> Circuit:
    b = _Builder(n)
    b.g1(H, 0)
    for i in range(n - 1):
        b.g2(CNOT, i, i + 1)
    return b.build()


def bell_pairs_circuit(n: int, pairs) -> Circuit:
    """Bell pairs (|00> + |11>)/sqrt2 between the listed qubit pairs, every
    other qubit left in |0>, with nearest-neighbour gates only: each pair is
    made on two adjacent qubits (H, CNOT), then adjacent SWAPs (a bubble sort)
    carry every qubit to its listed position."""
    pairs = [tuple(p) for p in pairs]
    used = [q for p in pairs for q in p]
    if len(set(used)) != len(used) or any(q < 0 or q >= n for q in used):
        raise ValueError("pairs must be disjoint qubits in range")
    free = [q for q in range(n) if q not in used]
    target = []                       # final position of the qubit at each start position
    for a, b in pairs:
        target += [a, b]
    target += free
    b = _Builder(n)
    for i in range(len(pairs)):
        b.g1(H, 2 * i)
        b.g2(CNOT, 2 * i, 2 * i + 1)
    t = list(target)
    changed = True
    while changed:
        changed = False
        for i in range(n - 1):
            if t[i] > t[i + 1]:
                b.g2(SWAP, i, i + 1)
                t[i], t[i + 1] = t[i + 1], t[i]
                changed = True
    return b.build()


def product_circuit(n: int, seed: int = 0) -> Circuit:
    rng = np.random.default_rng(seed)
    b = _Builder(n)
    for _ in range(3):
        for q in range(n):
            b.g1(int(rng.choice([H, S, T, X, Y, Z, X14, SQW])), q)
    return b.build()


# ---- random MPS states in right-canonical form -----------------------------
def bond_dims_saturated(n: int, chi: int) -> np.ndarray:
    """chi_b = min(chi, 2^b, 2^(n-b)) for bonds b = 0..n (boundaries are 1)."""
    b = np.arange(n + 1)
    lim = np.minimum(b, n - b).astype(np.int64)
    return np.minimum(chi, np.left_shift(1, np.minimum(lim, 40))).astype(np.int64)


def spectrum(chi: int, rng: np.random.Generator) -> np.ndarray:
    """Schmidt spectrum with sorted exponential (Porter-Thomas) weights, unit norm."""
    w = np.sort(rng.exponential(1.0, size=chi))[::-1]
    w = w / w.sum()
    return np.sqrt(w)


def random_right_canonical(n: int, chi: int, seed: int, dtype=np.complex128, chis=None):
    """Random MPS: Haar-random right isometries B_q (chi_q, 2, chi_{q+1}) and spectra.

    Returns (chi[n+1], sites list, lambdas list).  Rows of every
    B_q viewed as (chi_q, 2 chi_{q+1}) are orthonormal.  The spectra are drawn
    independently, so the stored lambdas are a synthetic stand-in for the
    Schmidt values of a saturated state (used for sizing and timing).
    """
    rng = np.random.default_rng(seed)
    chis = bond_dims_saturated(n, chi) if chis is None else np.asarray(chis, dtype=np.int64)
    sites, lams = [], []
    for q in range(n):
        cl, cr = int(chis[q]), int(chis[q + 1])
        g = rng.standard_normal((2 * cr, cl)) + 1j * rng.standard_normal((2 * cr, cl))
        qm, rm = np.linalg.qr(g)
        qm = qm * (np.diag(rm) / np.abs(np.diag(rm)))[None, :]
        sites.append(np.ascontiguousarray(qm.conj().T.reshape(cl, 2, cr)).astype(dtype))
    for bnd in range(n + 1):
        c = int(chis[bnd])
        lams.append(np.ones(1) if c == 1 else spectrum(c, rng))
    return chis, sites, lams


def random_right_canonical_device(n: int, chi: int, seed: int, device="cuda",
                                  dtype=None):
    """Device version of :func:`random_right_canonical` for large chi (torch).

    Same recipe: Gaussian (2 chi_r, chi_l) -> QR -> conjugate transpose.  The
    generator is torch's seeded device RNG, so values differ from the host
    version; shapes and distributions are the same.
    """
    import torch
    dtype = dtype or torch.complex64
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    chis = bond_dims_saturated(n, chi)
    sites = []
    for q in range(n):
        cl, cr = int(chis[q]), int(chis[q + 1])
        g = torch.randn((2 * cr, cl), dtype=dtype, device=device, generator=gen)
        qm, _ = torch.linalg.qr(g)
        sites.append(qm.conj().transpose(0, 1).contiguous().reshape(cl, 2, cr))
    rng = np.random.default_rng(seed)
    lams = [np.ones(1) if int(c) == 1 else spectrum(int(c), rng) for c in chis]
    return chis, sites, lams
