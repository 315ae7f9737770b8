"""FP64 reference of the surrogate network (TEST INFRASTRUCTURE).

Plain PyTorch CPU operations in float64 restating the network of
paper_2507_12610_gb300/surrogate.py layer by layer: its inputs, its three
message-passing rounds, its decoder and the mean-squared loss; gradients come
from autograd.  Only the tests use it.  It shares no code with the CUDA
kernels (it imports nothing from the package).
"""
from __future__ import annotations

import numpy as np
import torch

H, ROUNDS, OUT = 128, 3, 6


def features(x, v, w, R, off, nbr, vs, Rs):
    """Node and edge inputs (16 columns, column 7 = 1), float64."""
    n = len(R)
    nf = np.zeros((n, 16))
    nf[:, 0:3] = v / vs
    nf[:, 3:6] = R[:, None] * w / vs
    nf[:, 6] = R / Rs - 1.0
    nf[:, 7] = 1.0
    dst = np.repeat(np.arange(n), np.diff(off))
    d = x[nbr] - x[dst]
    ef = np.zeros((len(nbr), 16))
    ef[:, 0:3] = d / Rs
    ef[:, 3] = (np.linalg.norm(d, axis=1) - R[dst] - R[nbr]) / Rs
    ef[:, 4:7] = (v[nbr] - v[dst]) / vs
    ef[:, 7] = 1.0
    return nf, ef, dst


def neighbours(x, cutoff):
    """All pairs closer than cutoff: CSR by receiver, senders ascending."""
    d = np.linalg.norm(x[:, None] - x[None], axis=-1)
    n = len(x)
    mask = (d < cutoff) & ~np.eye(n, dtype=bool)
    off = np.concatenate([[0], np.cumsum(mask.sum(1))])
    nbr = np.nonzero(mask)[1]
    return off, nbr


def bf16(t):
    """Round to the nearest bfloat16 (ties to even), kept as float64."""
    return t.to(torch.bfloat16).to(torch.float64)


def forward(W: dict, nf, ef, dst, nbr, n, stored_bf16=False):
    """W: name -> float64 tensor [inputs incl. the constant column][outputs].

    stored_bf16: the network as the surrogate stores it, every layer input
    (node and edge features, the node states entering a layer, the edge
    states, the summed messages) rounded to bfloat16 where it is stored,
    the products and sums in float64 (the weights are passed rounded)."""
    relu = torch.relu
    r = bf16 if stored_bf16 else (lambda t: t)
    nf, ef = r(nf), r(ef)
    h = relu(nf @ W["node"])
    e = r(relu(ef @ W["edge"]))
    one = torch.zeros((e.shape[0], 16), dtype=torch.float64)
    one[:, 0] = 1.0
    onen = torch.zeros((n, 16), dtype=torch.float64)
    onen[:, 0] = 1.0
    for k in range(ROUNDS):
        hs = r(h)
        m = relu(torch.cat([hs[dst], hs[nbr], e, one], 1) @ W[f"msg{k}"])
        M = torch.zeros((n, H), dtype=torch.float64).index_add_(0, dst, m)
        h = h + relu(torch.cat([hs, r(M), onen], 1) @ W[f"upd{k}"])
    return torch.cat([r(h), onen], 1) @ W["dec"]


def loss_and_grads(weights: dict, nf, ef, dst, nbr, target):
    """Mean squared error over the n x 6 outputs and its gradients (float64)."""
    W = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in weights.items()}
    n = nf.shape[0]
    y = forward(W, torch.tensor(nf), torch.tensor(ef), torch.tensor(dst), torch.tensor(nbr), n)
    y = y[:, :OUT]
    loss = ((y - torch.tensor(target)) ** 2).mean()
    loss.backward()
    return float(loss.detach()), y.detach().numpy(), {k: W[k].grad.numpy() for k in W}
