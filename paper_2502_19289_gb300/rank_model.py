"""Training driver of the learned rank predictor that sizes the sketched split.

Pairs (features, retained rank) are logged from runs of the full split (no
sketch), the network is trained on the GPU with the library's own forward,
backward and Adam kernels (``mlp_loss_grad`` / ``mlp_adam``), and at
inference ``make_hint_fn`` turns its predicted rank bucket into the sketch
size hint of every split of an iteration (``rank_model_predict``).  The
target of a split is the bucket of r / B, r its rank after the cutoff and the
zero floor (before the chi_max cap) and B its Eq. 9 bound:
bucket b <=> r / B in (2^-(b+1)/2, 2^-b/2], b = 0..15.
"""
from __future__ import annotations

import math

import numpy as np

from . import (FP32, MPS, Circuit, cluster_partition, cluster_rank_bounds, cluster_unitary,
               make_config, mlp_adam, mlp_loss_grad, mlp_nparams, rank_features)

F, H1, H2, NB = 16, 64, 64, 16


def bucket_of(rank: np.ndarray, bound: np.ndarray) -> np.ndarray:
    ratio = np.clip(np.asarray(rank, float) / np.maximum(np.asarray(bound, float), 1.0), 1e-12, 1.0)
    return np.minimum(NB - 1, np.floor(-2.0 * np.log2(ratio) + 1e-9)).astype(np.int32)


def hint_of(bucket: np.ndarray, bound: np.ndarray) -> np.ndarray:
    return np.maximum(1, np.ceil(np.asarray(bound) * 2.0 ** (-0.5 * np.asarray(bucket)))).astype(np.int32)


def collect(circ_arrays, n_qubits, chi_max, cutoff, q_max, k_max, stream=None):
    """Run the full split over one circuit; return features, ranks, bounds."""
    circ = Circuit(n_qubits, *circ_arrays)
    cfg = make_config(n_qubits, chi_max, cutoff, q_max, 0, k_max, FP32)
    mps = MPS(cfg, stream)
    Xs, ranks, bounds = [], [], []
    start = 0
    while start < circ.n_layers:
        chi = mps.bond_dims()
        ent = mps.bond_entropies()
        clusters, stop = cluster_partition(circ.gates, circ.n_gates, start, chi, cfg)
        feats = {c.q0: rank_features(circ.gates, circ.n_gates, c, chi, ent, cfg) for c in clusters}
        bnds = {c.q0: cluster_rank_bounds(circ.gates, circ.n_gates, c, chi) for c in clusters}
        mps.apply_singletons(circ.gates, circ.n_gates, clusters, start, stop)
        if clusters:
            mps.step(clusters, [cluster_unitary(circ.gates, circ.n_gates, c) for c in clusters])
            for row in mps.split_log():
                q0, bond, r_eta = int(row[0]), int(row[2]), int(row[10])
                j = bond - q0
                Xs.append(feats[q0][j - 1])
                ranks.append(r_eta)
                bounds.append(int(bnds[q0][j - 1]))
        start = stop
    mps.close()
    if not Xs:
        return np.zeros((0, F), np.float32), np.zeros(0, np.int32), np.zeros(0, np.int32)
    return np.stack(Xs).astype(np.float32), np.array(ranks, np.int32), np.array(bounds, np.int32)


def init_params(seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    parts = []
    for fan_out, fan_in in ((H1, F), (H2, H1), (NB, H2)):
        parts.append(rng.standard_normal((fan_out, fan_in)).astype(np.float32) * math.sqrt(2.0 / fan_in))
        parts.append(np.zeros(fan_out, np.float32))
    p = np.concatenate([x.reshape(-1) for x in parts])
    assert p.size == mlp_nparams()
    return p


def train(X: np.ndarray, y: np.ndarray, epochs: int = 200, lr: float = 3e-3, batch: int = 512,
          seed: int = 0, device="cuda"):
    """Adam on the mean cross-entropy; every step runs the library's kernels.

    Returns (params, loss history per epoch)."""
    import torch
    n = mlp_nparams()
    dev = torch.device(device)
    P = torch.as_tensor(init_params(seed), device=dev)
    G = torch.zeros(n, device=dev)
    M1 = torch.zeros(n, device=dev)
    M2 = torch.zeros(n, device=dev)
    L = torch.zeros(1, device=dev)
    Xd = torch.as_tensor(np.ascontiguousarray(X, np.float32), device=dev)
    yd = torch.as_tensor(np.ascontiguousarray(y, np.int32), device=dev)
    rng = np.random.default_rng(seed)
    hist, t = [], 0
    N = len(y)
    for _ in range(epochs):
        perm = torch.as_tensor(rng.permutation(N), device=dev)
        tot = 0.0
        for s in range(0, N, batch):
            idx = perm[s:s + batch]
            xb = Xd[idx].contiguous()
            yb = yd[idx].contiguous()
            t += 1
            mlp_loss_grad(P.data_ptr(), xb.data_ptr(), yb.data_ptr(), len(idx), G.data_ptr(), L.data_ptr())
            mlp_adam(P.data_ptr(), G.data_ptr(), M1.data_ptr(), M2.data_ptr(), n, lr, t)
            tot += float(L.item()) * len(idx)
        hist.append(tot / max(N, 1))
    return P.cpu().numpy(), hist


def make_hint_fn(mps: MPS, circ: Circuit, cfg, params=None):
    """Hints for every split of an iteration from the loaded (or given) model."""
    if params is not None:
        mps.load_rank_model(params)

    def fn(clusters, chi):
        ent = mps.bond_entropies()
        rows, bnds, counts = [], [], []
        for c in clusters:
            rows.append(rank_features(circ.gates, circ.n_gates, c, chi, ent, cfg))
            bnds.append(cluster_rank_bounds(circ.gates, circ.n_gates, c, chi))
            counts.append(c.k - 1)
        if not rows:
            return []
        hints = mps.predict_hints(np.concatenate(rows), np.concatenate(bnds))
        out, o = [], 0
        for k1 in counts:
            out.append(hints[o:o + k1])
            o += k1
        return out

    return fn
