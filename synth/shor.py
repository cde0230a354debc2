"""Shor's factoring circuit in Beauregard's construction, as a gate list.

An input generator like the rest of ``synth``: it emits the gates of the
circuit the paper simulates in Sec. IV.B (order finding for a modulo N,
Beauregard's 2n + 3-qubit modular arithmetic with a full counting register),
restricted to the gate codes of ``synth`` and to nearest-neighbour two-qubit
gates.  It holds none of the simulation method's arithmetic.

Construction (Beauregard, "Circuit for Shor's algorithm using 2n+3 qubits",
Quantum Inf. Comput. 3, 175 (2003)), restated:

* registers on the chain, in this order: t counting qubits c, the n-qubit
  work register x (starts at |1>), the (n+1)-qubit addition register b
  (starts at |0>), one ancilla;
* QFT on b without the final reversal: qubit b_k ends with relative phase
  2 pi B / 2^(k+1) for the register value B = sum_k b_k 2^k;
* phi-ADD(a): a phase 2 pi a / 2^(k+1) on every b_k (addition of a
  constant modulo 2^(n+1) in the Fourier basis); controlled forms put each
  phase on a controlled or doubly controlled phase gate; a doubly controlled
  phase is CP(th/2)(c2, t) CNOT(c1, c2) CP(-th/2)(c2, t) CNOT(c1, c2)
  CP(th/2)(c1, t);
* phi-ADD(a)MOD(N): add a, subtract N, copy the sign bit (the top qubit of
  b, out of the Fourier basis) into the ancilla, add N back under the
  ancilla, then subtract a and use the sign bit once more to reset the
  ancilla, and add a again;
* CMULT(a)MOD(N): b <- b + a x mod N under control c, as n modular
  additions of 2^i a mod N, each controlled by c and x_i, inside a QFT of b;
* controlled U_a: CMULT(a), controlled swaps of x with the low n qubits of
  b, and the inverse of CMULT(a^-1 mod N);
* order finding: H on every counting qubit, controlled U_(a^(2^j)) by
  counting qubit c_j, then the inverse QFT on the counting register.  The
  inverse QFT is applied to the counting qubits in reverse order, so that
  measuring c_(t-1-k) gives bit k of the phase estimate y ~ s 2^t / r.

Routing (Sec. IV.B: long-range gates become chains of SWAP gates), two
variants.  "return" (the default): the counting qubit of each controlled U_a
is first moved next to the work register; every other two-qubit gate on
qubits further apart moves its first qubit next to its second, applies the
gate and moves it back.  Every qubit is back in place at the end, so the
circuit acts on the logical qubits in chain order.  "lazy": the same moves
without the returns; qubits end wherever the last gate left them, and
``shor_build`` reports where each register ended.  Every move is a chain of
nearest-neighbour SWAPs.
"""
from __future__ import annotations

import math

from . import CNOT, CP, SWAP, H, P, X, Circuit, _Builder


def counting_qubits(N: int, eps: float) -> int:
    """Counting-register size for phase estimation that succeeds with
    probability at least 1 - eps: t = 2n + 1 + ceil(log2(2 + 1 / (2 eps))),
    n = ceil(log2 N) (Nielsen and Chuang, Eq. 5.35)."""
    if not 0.0 < eps < 1.0:
        raise ValueError("eps must lie in (0, 1)")
    n = max(1, math.ceil(math.log2(N)))
    return 2 * n + 1 + math.ceil(math.log2(2.0 + 1.0 / (2.0 * eps)))


class _Router:
    """Emits logical gates on a chain through nearest-neighbour SWAPs.
    pos[l] is the chain position of logical qubit l, at[p] the logical qubit
    at position p.  lazy: a routed qubit stays where the gate needed it."""

    def __init__(self, n: int, lazy: bool = False):
        self.b = _Builder(n)
        self.pos = list(range(n))
        self.at = list(range(n))
        self.lazy = lazy

    def _swap(self, p: int):   # positions p and p + 1
        self.b.g2(SWAP, p, p + 1)
        u, v = self.at[p], self.at[p + 1]
        self.at[p], self.at[p + 1] = v, u
        self.pos[u], self.pos[v] = p + 1, p

    def move(self, l: int, target: int) -> list[int]:
        """Move logical qubit l to position target; returns the swaps done."""
        done = []
        while self.pos[l] < target:
            p = self.pos[l]
            self._swap(p)
            done.append(p)
        while self.pos[l] > target:
            p = self.pos[l] - 1
            self._swap(p)
            done.append(p)
        return done

    def undo(self, done: list[int]):
        if self.lazy:
            return
        for p in reversed(done):
            self._swap(p)

    def g1(self, kind: int, l: int, param: float = 0.0):
        self.b.g1(kind, self.pos[l], param)

    def g2(self, kind: int, la: int, lb: int, param: float = 0.0):
        pa, pb = self.pos[la], self.pos[lb]
        done = []
        if abs(pa - pb) > 1:
            done = self.move(la, pb - 1 if pa < pb else pb + 1)
        self.b.g2(kind, self.pos[la], self.pos[lb], param)
        self.undo(done)


class _Shor:
    def __init__(self, N: int, a: int, t: int, lazy: bool = False):
        if N < 3 or not (1 < a < N) or math.gcd(a, N) != 1:
            raise ValueError("need N >= 3 and 1 < a < N coprime to N")
        if t < 1:
            raise ValueError("need at least one counting qubit")
        self.N, self.a, self.t = N, a, t
        self.n = n = max(1, math.ceil(math.log2(N)))
        self.c = list(range(t))
        self.x = list(range(t, t + n))
        self.bq = list(range(t + n, t + 2 * n + 1))       # n + 1 qubits, bq[0] least significant
        self.anc = t + 2 * n + 1
        self.r = _Router(t + 2 * n + 2, lazy)

    # -- Fourier-basis arithmetic on b ------------------------------------
    def qft(self, qs, inverse=False):
        """In-place QFT without the final reversal on qubits qs (qs[0] least
        significant): qubit qs[k] ends with phase 2 pi B / 2^(k+1)."""
        ops = []
        for k in range(len(qs) - 1, -1, -1):
            ops.append(("h", qs[k], None, 0.0))
            for j in range(k - 1, -1, -1):
                ops.append(("cp", qs[j], qs[k], math.pi / (1 << (k - j))))
        if inverse:
            ops = [(o, u, v, -th) for (o, u, v, th) in reversed(ops)]
        for o, u, v, th in ops:
            if o == "h":
                self.r.g1(H, u)
            else:
                self.r.g2(CP, u, v, th)

    def _phase(self, ctrls, q, th):
        """Phase th on |1> of q, controlled by 0, 1 or 2 qubits."""
        if abs(math.remainder(th, 2.0 * math.pi)) < 1e-15:
            return
        if not ctrls:
            self.r.g1(P, q, th)
        elif len(ctrls) == 1:
            self.r.g2(CP, ctrls[0], q, th)
        else:
            c1, c2 = ctrls
            self.r.g2(CP, c2, q, th / 2)
            self.r.g2(CNOT, c1, c2)
            self.r.g2(CP, c2, q, -th / 2)
            self.r.g2(CNOT, c1, c2)
            self.r.g2(CP, c1, q, th / 2)

    def phi_add(self, a, ctrls=(), sign=1):
        """b <- b + sign * a (mod 2^(n+1)) in the Fourier basis."""
        for k, q in enumerate(self.bq):
            self._phase(list(ctrls), q, sign * 2.0 * math.pi * a / (1 << (k + 1)))

    def phi_add_mod(self, a, c1, c2, inverse=False):
        """b <- b + a mod N when c1 = c2 = 1 (b < N), Fourier basis in and out;
        the ancilla starts and ends at |0>."""
        N, top, anc = self.N, self.bq[-1], self.anc
        steps = [
            lambda s: self.phi_add(a, (c1, c2), s),
            lambda s: self.phi_add(N, (), -s),
            lambda s: self.qft(self.bq, inverse=True),
            lambda s: self.r.g2(CNOT, top, anc),
            lambda s: self.qft(self.bq),
            lambda s: self.phi_add(N, (anc,), s),
            lambda s: self.phi_add(a, (c1, c2), -s),
            lambda s: self.qft(self.bq, inverse=True),
            lambda s: self.r.g1(X, top),
            lambda s: self.r.g2(CNOT, top, anc),
            lambda s: self.r.g1(X, top),
            lambda s: self.qft(self.bq),
            lambda s: self.phi_add(a, (c1, c2), s),
        ]
        if not inverse:
            for f in steps:
                f(1)
            return
        # the inverse: steps in reverse order, each inverted (the QFTs swap
        # with their inverses; X and CNOT are their own inverses)
        inv = {2: lambda: self.qft(self.bq), 4: lambda: self.qft(self.bq, inverse=True),
               7: lambda: self.qft(self.bq), 11: lambda: self.qft(self.bq, inverse=True)}
        for i in range(len(steps) - 1, -1, -1):
            if i in inv:
                inv[i]()
            else:
                steps[i](-1)

    def cmult(self, a, c, inverse=False):
        """b <- b + a x mod N under control c (inverse: b <- b - a x mod N)."""
        self.qft(self.bq)
        idx = range(self.n - 1, -1, -1) if inverse else range(self.n)
        for i in idx:
            self.phi_add_mod((a << i) % self.N, c, self.x[i], inverse=inverse)
        self.qft(self.bq, inverse=True)

    def cswap(self, c, u, v):
        """Controlled swap of u and v: CNOT(v, u) Toffoli(c, u; v) CNOT(v, u),
        the Toffoli as H(v) CCZ H(v) with CCZ = doubly controlled phase pi."""
        self.r.g2(CNOT, v, u)
        self.r.g1(H, v)
        self._phase([c, u], v, math.pi)
        self.r.g1(H, v)
        self.r.g2(CNOT, v, u)

    def controlled_u(self, a, cj):
        """x <- a x mod N under control cj (b and the ancilla stay |0>)."""
        # bring the control next to the work register for the whole block
        px = self.r.pos[self.x[0]]
        done = self.r.move(cj, px - 1 if self.r.pos[cj] < px else px + 1)
        self.cmult(a, cj)
        for i in range(self.n):
            self.cswap(cj, self.x[i], self.bq[i])
        self.cmult(pow(a, -1, self.N), cj, inverse=True)
        self.r.undo(done)

    def build(self) -> Circuit:
        for q in self.c:
            self.r.g1(H, q)
        self.r.g1(X, self.x[0])
        for j in range(self.t):
            self.controlled_u(pow(self.a, 1 << j, self.N), self.c[j])
        # inverse QFT with counting qubit c_j as the weight-2^(t-1-j) bit
        self.qft(list(reversed(self.c)), inverse=True)
        return self.r.b.build()


def shor_build(N: int, a: int, t: int | None = None, eps: float = 1e-3,
               routing: str = "return") -> tuple[Circuit, dict]:
    """Order finding of a modulo N with t counting qubits (default from eps,
    see ``counting_qubits``): t + 2n + 2 qubits; nearest-neighbour gates only.
    Returns the circuit and the chain positions its registers end at: "c"
    (counting qubit c_j at c[j]), "x" (x_0 least significant), "b" (b_0
    least significant), "anc".  With routing "return" they are the start
    positions, in that order along the chain."""
    if routing not in ("return", "lazy"):
        raise ValueError("routing is 'return' or 'lazy'")
    sh = _Shor(N, a, counting_qubits(N, eps) if t is None else t, lazy=routing == "lazy")
    circ = sh.build()
    pos = sh.r.pos
    regs = {"c": [pos[q] for q in sh.c], "x": [pos[q] for q in sh.x], "b": [pos[q] for q in sh.bq],
            "anc": pos[sh.anc]}
    return circ, regs


def shor_circuit(N: int, a: int, t: int | None = None, eps: float = 1e-3) -> Circuit:
    """``shor_build`` with routing "return": chain order counting register,
    work register x, addition register b, ancilla."""
    return shor_build(N, a, t, eps)[0]


def shor_registers(N: int, t: int) -> dict:
    """Chain positions of the registers of ``shor_circuit(N, a, t)``."""
    n = max(1, math.ceil(math.log2(N)))
    return {"c": list(range(t)), "x": list(range(t, t + n)),
            "b": list(range(t + n, t + 2 * n + 1)), "anc": t + 2 * n + 1}
