"""Pins of the FP64 reference of the surrogate network (CPU)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
mo = pytest.importorskip("oracle.mpnn_oracle")

SHAPES = {"node": (16, 128), "edge": (16, 128), "dec": (144, 64)}
for r in range(3):
    SHAPES[f"msg{r}"] = (400, 128)
    SHAPES[f"upd{r}"] = (272, 128)


def small_case(seed=0, n=7):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 4e-3, size=(n, 3))
    v = rng.normal(scale=0.1, size=(n, 3))
    w = rng.normal(scale=20.0, size=(n, 3))
    R = rng.uniform(0.9e-3, 1.1e-3, size=n)
    off, nbr = mo.neighbours(x, 2.6e-3)
    nf, ef, dst = mo.features(x, v, w, R, off, nbr, 0.1, 1e-3)
    W = {k: rng.normal(scale=0.3 / np.sqrt(s[0]), size=s) for k, s in SHAPES.items()}
    W["dec"][:, 6:] = 0.0
    T = rng.normal(size=(n, 6))
    return W, nf, ef, dst, nbr, T


def test_gradients_match_central_differences():
    W, nf, ef, dst, nbr, T = small_case()
    assert len(nbr) > 6
    loss, _, G = mo.loss_and_grads(W, nf, ef, dst, nbr, T)
    rng = np.random.default_rng(1)
    for name in SHAPES:
        rows, cols = SHAPES[name]
        for _ in range(3):
            i, j = int(rng.integers(rows)), int(rng.integers(min(cols, 6 if name == "dec" else cols)))
            h = 1e-6
            Wp = {k: v.copy() for k, v in W.items()}
            Wm = {k: v.copy() for k, v in W.items()}
            Wp[name][i, j] += h
            Wm[name][i, j] -= h
            fd = (mo.loss_and_grads(Wp, nf, ef, dst, nbr, T)[0]
                  - mo.loss_and_grads(Wm, nf, ef, dst, nbr, T)[0]) / (2 * h)
            assert G[name][i, j] == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, i, j)


def test_outputs_follow_a_relabelling_of_the_particles():
    W, nf, ef, dst, nbr, T = small_case(seed=3)
    rng = np.random.default_rng(4)
    # rebuild from a permuted particle set
    n = nf.shape[0]
    p = rng.permutation(n)
    x = rng.uniform(0, 4e-3, size=(n, 3))
    v = rng.normal(scale=0.1, size=(n, 3))
    w = rng.normal(scale=20.0, size=(n, 3))
    R = rng.uniform(0.9e-3, 1.1e-3, size=n)
    outs = []
    for perm in (np.arange(n), p):
        off, nb = mo.neighbours(x[perm], 2.6e-3)
        a, b, d = mo.features(x[perm], v[perm], w[perm], R[perm], off, nb, 0.1, 1e-3)
        outs.append(mo.loss_and_grads(W, a, b, d, nb, np.zeros((n, 6)))[1])
    inv = np.argsort(p)
    assert np.allclose(outs[1][inv], outs[0], rtol=1e-12, atol=1e-15)


def test_decoder_bias_alone_is_the_output():
    W, nf, ef, dst, nbr, T = small_case(seed=5)
    W = {k: np.zeros_like(v) for k, v in W.items()}
    b = np.array([0.5, -1.0, 2.0, 0.25, 0.0, -0.75])
    W["dec"][128, :6] = b
    _, y, _ = mo.loss_and_grads(W, nf, ef, dst, nbr, T)
    assert np.array_equal(y, np.tile(b, (nf.shape[0], 1)))


def test_stored_bf16_forward_rounds_only_where_it_stores():
    # on values that bfloat16 holds exactly rounding the stored layer inputs
    # changes nothing; on general values it moves the output by about
    # bfloat16's relative precision, not more
    W, nf, ef, dst, nbr, T = small_case(seed=3)
    n = nf.shape[0]
    args = (torch.tensor(dst), torch.tensor(nbr), n)
    Wt = {k: torch.tensor(v) for k, v in W.items()}
    y = mo.forward(Wt, torch.tensor(nf), torch.tensor(ef), *args)
    yb = mo.forward(Wt, torch.tensor(nf), torch.tensor(ef), *args, stored_bf16=True)
    rel = float((yb - y).abs().max() / y.abs().max())
    assert 1e-5 < rel < 5e-2, rel
    # exact case: every layer output copies one of its inputs (one weight 1
    # per output column), features are 0, 1 or 2, messages copy edge states
    # or the constant, so every value is an integer far below 256
    rng = np.random.default_rng(5)
    H = mo.H

    def copies(kin, kout, lo=0, hi=None):
        w = np.zeros((kin, kout))
        w[rng.integers(lo, hi if hi is not None else kin, size=kout), np.arange(kout)] = 1.0
        return torch.tensor(w)

    Wi = {"node": copies(16, H), "edge": copies(16, H), "dec": copies(H + 16, 64)}
    for r in range(3):
        Wi[f"msg{r}"] = copies(3 * H + 16, H, 2 * H, 3 * H + 1)  # edge states or the constant
        Wi[f"upd{r}"] = copies(2 * H + 16, H, 0, 2 * H + 1)
    nfi = torch.tensor(rng.integers(0, 3, size=nf.shape).astype(np.float64))
    efi = torch.tensor(rng.integers(0, 3, size=ef.shape).astype(np.float64))
    y0 = mo.forward(Wi, nfi, efi, *args)
    y1 = mo.forward(Wi, nfi, efi, *args, stored_bf16=True)
    assert 0 < float(y0.abs().max()) < 256
    assert torch.equal(y0, y1)
