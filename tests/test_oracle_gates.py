"""Pins for the oracle's gate tables (App. A) and state-vector simulator (Sec. II.A)."""
import math
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "appA_gates.txt")
NAME2KIND = {"H": synth.H, "X": synth.X, "Y": synth.Y, "Z": synth.Z, "T": synth.T,
             "CNOT": synth.CNOT, "CY": synth.CY, "CZ": synth.CZ, "SWAP": synth.SWAP,
             "CH": synth.CH, "CS": synth.CS, "CT": synth.CT, "SQSWAP": synth.SQSWAP}


def _num(tok):
    env = {"r": 1 / math.sqrt(2), "pi": math.pi, "cos": math.cos, "sin": math.sin}
    tok = tok.replace("3pi", "3*pi")
    return float(eval(tok, {"__builtins__": {}}, env))


def _golden():
    out = {}
    for line in open(GOLD):
        if not line.strip() or line.startswith("#"):
            continue
        parts = line.split()
        name, d = parts[0], int(parts[1])
        vals = [complex(_num(a), _num(b)) for a, b in (p.split(",") for p in parts[2:])]
        out[name] = np.array(vals).reshape(d, d)
    return out


def test_printed_matrices_match_appendix():
    gold = _golden()
    for name, M in gold.items():
        if name == "P3PI4":
            got = oracle.gate_matrix(synth.P, 3 * math.pi / 4)
        else:
            got = oracle.gate_matrix(NAME2KIND[name])
        np.testing.assert_allclose(got, M, atol=1e-15, err_msg=name)


@pytest.mark.parametrize("kind", synth.ONE_QUBIT + synth.TWO_QUBIT)
def test_unitary(kind):
    U = oracle.gate_matrix(kind, 0.37)
    np.testing.assert_allclose(U.conj().T @ U, np.eye(U.shape[0]), atol=1e-14)


def test_algebraic_identities():
    g = oracle.gate_matrix
    X, Y, Z, H, S, T = (g(k) for k in (synth.X, synth.Y, synth.Z, synth.H, synth.S, synth.T))
    np.testing.assert_allclose(np.linalg.matrix_power(g(synth.X14), 4), X, atol=1e-14)
    np.testing.assert_allclose(g(synth.SQW) @ g(synth.SQW), (X + Y) / math.sqrt(2), atol=1e-14)
    np.testing.assert_allclose(g(synth.SQSWAP) @ g(synth.SQSWAP), g(synth.SWAP), atol=1e-14)
    np.testing.assert_allclose(T @ T, S, atol=1e-15)
    np.testing.assert_allclose(S @ S, Z, atol=1e-15)
    np.testing.assert_allclose(H @ Z @ H, X, atol=1e-15)
    np.testing.assert_allclose(g(synth.P, math.pi / 4), T, atol=1e-15)
    # controlled gates are |0><0| (x) I + |1><1| (x) G with the first qubit as control
    P0, P1 = np.diag([1, 0]), np.diag([0, 1])
    for ck, t in ((synth.CNOT, X), (synth.CY, Y), (synth.CZ, Z), (synth.CH, H), (synth.CS, S),
                  (synth.CT, T)):
        np.testing.assert_allclose(g(ck), np.kron(P0, np.eye(2)) + np.kron(P1, t), atol=1e-15)


def _kron_unitary(n, gates, params):
    """Independent construction: full 2^n unitary from np.kron (n <= 6)."""
    U = np.eye(1 << n, dtype=complex)
    for (nq, q0, q1, _q2, kind), p in zip(gates, params):
        G = oracle.gate_matrix(kind, p)
        if nq == 1:
            ops = [np.eye(2)] * n
            ops[q0] = G
            full = ops[0]
            for o in ops[1:]:
                full = np.kron(full, o)
        else:
            # embed on (q0,q1) by permuting a kron on adjacent (0,1)
            full = np.kron(G, np.eye(1 << (n - 2)))
            perm = [q0, q1] + [q for q in range(n) if q not in (q0, q1)]
            full = full.reshape([2] * (2 * n))
            inv = np.argsort(perm)
            full = full.transpose(list(inv) + [n + i for i in inv]).reshape(1 << n, 1 << n)
        U = full @ U
    return U


@pytest.mark.parametrize("seed", range(5))
def test_statevector_against_kron(seed):
    rng = np.random.default_rng(seed)
    n = 5
    rows, params = [], []
    for _ in range(25):
        if rng.random() < 0.5:
            rows.append((1, int(rng.integers(n)), -1, -1, int(rng.choice(synth.ONE_QUBIT))))
        else:
            a, b = rng.choice(n, 2, replace=False)  # any order, not only adjacent
            rows.append((2, int(a), int(b), -1, int(rng.choice(synth.TWO_QUBIT))))
        params.append(float(rng.uniform(0, 2 * np.pi)))
    circ = synth.Circuit(n, np.array(rows, dtype=np.int32), np.array(params))
    psi = oracle.statevector(circ)
    ref = _kron_unitary(n, rows, params)[:, 0]
    np.testing.assert_allclose(psi, ref, atol=1e-13)


def test_big_endian_basis():
    # X on qubit 0 of 3 qubits gives |100> = index 4 (qubit 0 is the MSB).
    circ = synth.Circuit(3, np.array([[1, 0, -1, -1, synth.X]], np.int32), np.zeros(1))
    psi = oracle.statevector(circ)
    assert abs(psi[4] - 1) < 1e-15
