"""Learned surrogate: a message-passing network over the particle neighbour
graph that predicts each particle's mean linear and angular acceleration
over a stride of DEM steps, trained on trajectories of the GPU DEM itself,
with the DEM as its fallback and as the judge of its error.

Network (hidden width 128, bf16 weights, fp32 accumulation; every layer's
bias is carried by a constant-1 input column):
  node encoder   h  = relu([node features, 1] W_n)                 16 -> 128
  edge encoder   e  = relu([edge features, 1] W_e)                 16 -> 128
  3 rounds       m_ij = relu([h_i, h_j, e_ij, 1] W_m)             400 -> 128
                 M_i  = sum over neighbours j of m_ij (receiver i)
                 h_i += relu([h_i, M_i, 1] W_u)                    272 -> 128
  decoder        y_i = [h_i, 1] W_d   (6 outputs: a_i, R_i alpha_i) 144 -> 6
The neighbour graph joins particles closer than 2.2 R_max.  Every matrix
product, gather, segment sum, transpose, loss and Adam update runs in the
kernels of mpnn.cu (include/mpnn.h); this module only allocates buffers
(PyTorch device memory) and sequences the calls.  Sums follow the graph's
CSR order, so forward and backward passes are deterministic.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import dem as _dem

EXPORTS = ("mpnn_gemm", "mpnn_gemm_split", "mpnn_transpose_bf16", "mpnn_to_bf16",
           "mpnn_graph", "mpnn_graph_cells", "mpnn_reverse_edges", "mpnn_features", "mpnn_gather_edges",
           "mpnn_concat_rows", "mpnn_residual", "mpnn_gather_rows", "mpnn_segment_sum",
           "mpnn_segment_sum_cols", "mpnn_segment_sum_perm", "mpnn_relu_backward",
           "mpnn_adam", "mpnn_mse")

H = 128          # hidden width
ROUNDS = 3       # message-passing rounds
OUT = 6          # a (3), R alpha (3)
# (inputs incl. the constant column, outputs) per layer
LAYERS = {"node": (16, H), "edge": (16, H), "dec": (H + 16, 64)}
for _r in range(ROUNDS):
    LAYERS[f"msg{_r}"] = (3 * H + 16, H)
    LAYERS[f"upd{_r}"] = (2 * H + 16, H)


def pad64(n: int) -> int:
    return max(64, (n + 63) // 64 * 64)


_lib = None


def load():
    global _lib
    if _lib is None:
        lib = _dem.load()
        for name in EXPORTS:
            getattr(lib, name).restype = ctypes.c_int
        _lib = lib
    return _lib


def _call(name, *args):
    conv = []
    for a in args:
        if isinstance(a, float):
            conv.append(ctypes.c_float(a))
        elif isinstance(a, bool):
            conv.append(ctypes.c_int32(int(a)))
        elif isinstance(a, int):
            conv.append(ctypes.c_int64(a))
        elif a is None:
            conv.append(ctypes.c_void_p(0))
        elif isinstance(a, (ctypes._SimpleCData, ctypes._Pointer)):
            conv.append(a)
        else:  # a torch tensor
            conv.append(ctypes.c_void_p(a.data_ptr()))
    rc = getattr(load(), name)(*conv)
    if rc != 0:
        raise _dem.DemError(rc, name)


def _i32(v):
    return ctypes.c_int32(int(v))


class Graph:
    """Neighbour graph and network inputs for one particle state (device)."""

    # cells the cell-list graph may use (workspace 2 x 8 B per cell)
    MAX_CELLS = 1 << 24

    def __init__(self, x, v, w, R, cutoff, vs, Rs, max_edges=None, all_pairs=False):
        import torch
        dev = torch.device("cuda")
        n = int(R.shape[0])
        self.n, self.npad = n, pad64(n)
        f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device=dev)
        self.x, self.v, self.w, self.R = f32(x), f32(v), f32(w), f32(R)
        cnt = torch.empty(n, dtype=torch.int64, device=dev)
        self.off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        ne = ctypes.c_int64(0)
        cap = max_edges or 64 * n
        self.nbr = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        self.dst = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        if all_pairs:  # O(n^2), kept as the reference of the cell-list graph
            _call("mpnn_graph", n, self.x, float(cutoff), cnt, self.off, self.nbr, self.dst, cap,
                  ctypes.pointer(ne), None)
        else:
            work = torch.empty(2 * (self.MAX_CELLS + 1) + 2 * n + 1, dtype=torch.int64,
                               device=dev)
            box = torch.empty(6, dtype=torch.float32, device=dev)
            _call("mpnn_graph_cells", n, self.x, float(cutoff), self.MAX_CELLS, work, box, cnt,
                  self.off, self.nbr, self.dst, cap, ctypes.pointer(ne), None)
        self.E = int(ne.value)
        self.Epad = pad64(self.E)
        self.perm = torch.empty(max(self.E, 1), dtype=torch.int32, device=dev)
        _call("mpnn_reverse_edges", self.E, self.off, self.nbr, self.dst, self.perm, None)
        self.nf = torch.empty(self.npad * 16, dtype=torch.int16, device=dev)
        self.ef = torch.empty(self.Epad * 16, dtype=torch.int16, device=dev)
        _call("mpnn_features", n, self.npad, self.E, self.Epad, self.dst, self.nbr, self.x,
              self.v, self.w, self.R, float(vs), float(Rs), self.nf, self.ef, None)
        # identity offsets: a one-row "segment" per node / per edge (column copies)
        self.ident_n = torch.arange(self.npad + 1, dtype=torch.int64, device=dev)
        self.ident_e = torch.arange(self.Epad + 1, dtype=torch.int64, device=dev)

    def edges_host(self):
        off = self.off.cpu().numpy()
        return off, self.nbr[:self.E].cpu().numpy(), self.dst[:self.E].cpu().numpy()


class MPNN:
    """The network's parameters (fp32 masters, bf16 copies, Adam moments)."""

    def __init__(self, seed=0, weights=None):
        import torch
        self.torch = torch
        dev = torch.device("cuda")
        rng = np.random.default_rng(seed)
        self.W, self.Wb, self.Wt, self.m, self.v, self.G = {}, {}, {}, {}, {}, {}
        for name, (kin, nout) in LAYERS.items():
            kp = pad64(kin)
            if weights is not None:
                w = np.zeros((kp, nout), np.float32)
                w[:kin] = weights[name]
            else:
                w = np.zeros((kp, nout), np.float32)
                cols = nout if name != "dec" else OUT
                if kin == 16:   # input layers: 7 features, the constant in column 7
                    w[:7] = rng.normal(scale=math.sqrt(2.0 / 7), size=(7, nout))
                    w[7] = 0.1
                else:           # hidden inputs, then the constant block
                    scale = math.sqrt(2.0 / (kin - 16)) if name != "dec" else 0.1 / math.sqrt(kin)
                    w[:kin - 16, :cols] = rng.normal(scale=scale, size=(kin - 16, cols))
            self.W[name] = torch.as_tensor(w, device=dev)
            self.Wb[name] = torch.empty((kp, nout), dtype=torch.int16, device=dev)
            self.Wt[name] = torch.empty((nout, kin), dtype=torch.int16, device=dev)
            self.m[name] = torch.zeros_like(self.W[name])
            self.v[name] = torch.zeros_like(self.W[name])
            self.G[name] = torch.zeros_like(self.W[name])
            self._refresh(name)
        self.t = 0
        self.zero_bias = torch.zeros(256, dtype=torch.float32, device=dev)

    def _refresh(self, name):
        # bf16 copies through a zero-rate Adam step would move the moments;
        # convert directly instead
        kin, nout = LAYERS[name]
        W = self.W[name]
        _call("mpnn_to_bf16", W.numel(), W, self.Wb[name], None)
        Wt32 = W[:kin].t().contiguous()
        _call("mpnn_to_bf16", Wt32.numel(), Wt32, self.Wt[name], None)

    def weights(self) -> dict:
        return {k: self.W[k][:LAYERS[k][0]].cpu().numpy().astype(np.float64) for k in LAYERS}

    # ---- forward -------------------------------------------------------------
    def forward(self, g: Graph, keep=True):
        torch = self.torch
        dev = torch.device("cuda")
        n, npad, E, Epad = g.n, g.npad, g.E, g.Epad
        st = {}
        z = self.zero_bias

        def gemm(M, N, K, A, name, relu, C=None, Cb=None):
            C = torch.empty((M, N), dtype=torch.float32, device=dev) if C is None else C
            _call("mpnn_gemm", M, N, K, A, self.Wt[name], C, Cb, z, _i32(2 if relu else 0),
                  _i32(0), None)
            return C

        hb = torch.empty((npad, H), dtype=torch.int16, device=dev)
        h = gemm(npad, H, 16, g.nf, "node", True, Cb=hb)
        st["h0"] = h.clone()
        eb = torch.empty((Epad, H), dtype=torch.int16, device=dev)
        e = gemm(Epad, H, 16, g.ef, "edge", True, Cb=eb)
        st["e"] = e
        for r in range(ROUNDS):
            Xm = torch.empty((Epad, 3 * H + 16), dtype=torch.int16, device=dev)
            _call("mpnn_gather_edges", E, Epad, _i32(H), _i32(H), g.dst, g.nbr, hb, eb, Xm, None)
            m = gemm(Epad, H, 3 * H + 16, Xm, f"msg{r}", True)
            Mi = torch.empty((npad, H), dtype=torch.float32, device=dev)
            _call("mpnn_segment_sum", n, npad, _i32(H), g.off, m, Mi, None)
            Xu = torch.empty((npad, 2 * H + 16), dtype=torch.int16, device=dev)
            _call("mpnn_concat_rows", n, npad, _i32(H), _i32(H), hb, Mi, Xu, None)
            u = gemm(npad, H, 2 * H + 16, Xu, f"upd{r}", True)
            _call("mpnn_residual", npad * H, h, u, hb, None)
            if keep:
                st[f"Xm{r}"], st[f"m{r}"], st[f"Xu{r}"], st[f"u{r}"] = Xm, m, Xu, u
        Xd = torch.empty((npad, H + 16), dtype=torch.int16, device=dev)
        _call("mpnn_concat_rows", n, npad, _i32(H), _i32(0), hb, None, Xd, None)
        y = gemm(npad, 64, H + 16, Xd, "dec", False)
        st["Xd"] = Xd
        self.state = st if keep else None
        return y

    # ---- backward ------------------------------------------------------------
    def _wgrad(self, name, X, rows, dZ):
        """G[name] = X^T dZ with X (bf16 [rows][kin]) and dZ (fp32 [rows][N])."""
        torch = self.torch
        dev = torch.device("cuda")
        kin, nout = LAYERS[name]
        kp = pad64(kin)
        XT = torch.zeros((kp, rows), dtype=torch.int16, device=dev)
        _call("mpnn_transpose_bf16", kin, rows, X, XT, None)
        dZb = torch.empty((rows, nout), dtype=torch.int16, device=dev)
        _call("mpnn_to_bf16", rows * nout, dZ, dZb, None)
        dZT = torch.empty((nout, rows), dtype=torch.int16, device=dev)
        _call("mpnn_transpose_bf16", nout, rows, dZb, dZT, None)
        splits = max(1, min(64, rows // 4096))
        work = torch.empty((splits, kp, nout), dtype=torch.float32, device=dev)
        _call("mpnn_gemm_split", kp, nout, rows, _i32(splits), XT, dZT, self.G[name], _i32(0),
              work, None)
        return dZb

    def _dx(self, name, dZb, rows):
        """dX = dZ W^T: fp32 [rows][pad64(kin)]."""
        torch = self.torch
        kin, nout = LAYERS[name]
        kp = pad64(kin)
        dX = torch.empty((rows, kp), dtype=torch.float32, device=torch.device("cuda"))
        _call("mpnn_gemm", rows, kp, nout, dZb, self.Wb[name], dX, None, None, _i32(0), _i32(0),
              None)
        return dX

    def backward(self, g: Graph, dy):
        torch = self.torch
        dev = torch.device("cuda")
        st = self.state
        n, npad, E, Epad = g.n, g.npad, g.E, g.Epad
        dyb = self._wgrad("dec", st["Xd"], npad, dy)
        dXd = self._dx("dec", dyb, npad)
        dh = torch.empty((npad, H), dtype=torch.float32, device=dev)
        _call("mpnn_segment_sum_cols", npad, npad, _i32(H), dXd.shape[1], _i32(0), g.ident_n,
              None, dXd, dh, None)
        de = torch.zeros((Epad, H), dtype=torch.float32, device=dev)
        tmp_b = torch.empty((max(npad, Epad) * H,), dtype=torch.int16, device=dev)
        for r in reversed(range(ROUNDS)):
            du = dh.clone()
            _call("mpnn_relu_backward", npad * H, st[f"u{r}"], du, None)
            dub = self._wgrad(f"upd{r}", st[f"Xu{r}"], npad, du)
            dXu = self._dx(f"upd{r}", dub, npad)
            w = dXu.shape[1]
            part = torch.empty((npad, H), dtype=torch.float32, device=dev)
            _call("mpnn_segment_sum_cols", npad, npad, _i32(H), w, _i32(0), g.ident_n, None, dXu,
                  part, None)
            _call("mpnn_residual", npad * H, dh, part, tmp_b, None)   # dh += d/dh of [h, M]
            dM = torch.empty((npad, H), dtype=torch.float32, device=dev)
            _call("mpnn_segment_sum_cols", npad, npad, _i32(H), w, _i32(H), g.ident_n, None, dXu,
                  dM, None)
            dm = torch.empty((Epad, H), dtype=torch.float32, device=dev)
            _call("mpnn_gather_rows", E, Epad, _i32(H), g.dst, dM, dm, None)
            _call("mpnn_relu_backward", Epad * H, st[f"m{r}"], dm, None)
            dmb = self._wgrad(f"msg{r}", st[f"Xm{r}"], Epad, dm)
            dXm = self._dx(f"msg{r}", dmb, Epad)
            w = dXm.shape[1]
            _call("mpnn_segment_sum_cols", n, npad, _i32(H), w, _i32(0), g.off, None, dXm, part,
                  None)
            _call("mpnn_residual", npad * H, dh, part, tmp_b, None)   # receivers
            _call("mpnn_segment_sum_cols", n, npad, _i32(H), w, _i32(H), g.off, g.perm, dXm,
                  part, None)
            _call("mpnn_residual", npad * H, dh, part, tmp_b, None)   # senders
            pe = torch.empty((Epad, H), dtype=torch.float32, device=dev)
            _call("mpnn_segment_sum_cols", Epad, Epad, _i32(H), w, _i32(2 * H), g.ident_e, None,
                  dXm, pe, None)
            _call("mpnn_residual", Epad * H, de, pe, tmp_b, None)     # edge embeddings
        _call("mpnn_relu_backward", Epad * H, st["e"], de, None)
        self._wgrad("edge", g.ef, Epad, de)
        _call("mpnn_relu_backward", npad * H, st["h0"], dh, None)
        self._wgrad("node", g.nf, npad, dh)

    def loss_and_grad(self, g: Graph, target):
        """MSE over the n x 6 outputs; target fp32 [npad][64] (zeros past 6
        columns and n rows).  Fills G and returns the loss."""
        torch = self.torch
        dev = torch.device("cuda")
        y = self.forward(g)
        dy = torch.empty_like(y)
        out = torch.zeros(1, dtype=torch.float32, device=dev)
        _call("mpnn_mse", y.numel(), y, target, 1.0 / (g.n * OUT), dy, out, None)
        self.backward(g, dy)
        return float(out.item()) / (g.n * OUT)

    def adam(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        for name, (kin, nout) in LAYERS.items():
            W = self.W[name]
            _call("mpnn_adam", W.numel(), W, self.m[name], self.v[name], self.G[name], float(lr),
                  float(b1), float(b2), float(eps), self.t, self.Wb[name], self.Wt[name],
                  _i32(W.shape[0]), _i32(nout), _i32(kin), None)


# ---- data from the DEM ---------------------------------------------------------

def targets(v0, w0, v1, w1, R, stride, dt, a_s):
    """Mean accelerations over the stride, scaled: [a, R alpha] / a_s."""
    a = (v1 - v0) / (stride * dt)
    al = (w1 - w0) / (stride * dt) * R[:, None]
    return np.hstack([a, al]) / a_s


def target_buffer(T, npad):
    import torch
    buf = np.zeros((npad, 64), np.float32)
    buf[:T.shape[0], :OUT] = T
    return torch.as_tensor(buf, device=torch.device("cuda"))


SCALES = dict(vs=0.1, Rs=1.0e-3, a_s=10.0)   # velocity, length, acceleration scales


def make_graph(x, v, w, R, rmax):
    return Graph(x, v, w, R, 2.2 * rmax, SCALES["vs"], SCALES["Rs"])


def sample_pairs(scene, n_samples, every=50, stride=10, settle=2000, precision=1):
    """(state at t, state at t + stride) pairs from a GPU DEM run of `scene`
    (dict for dem.Scene.from_dict): settle, then a pair every `every` steps."""
    sc = _dem.Scene.from_dict(scene, precision=precision)
    sc.step(settle)
    R = sc.radii()
    out = []
    for _ in range(n_samples):
        a = sc.state()
        sc.step(stride)
        b = sc.state()
        out.append((a, b))
        sc.step(max(0, every - stride))
    if sc.synchronize() != 0:
        raise RuntimeError("DEM run failed")
    return out, R


def train(model: MPNN, pairs, R, dt, stride=10, iters=300, lr=1e-3, log_every=50, lr_end=None):
    """Adam on the mean-squared error of the scaled mean accelerations,
    cycling through the sample pairs (learning rate decaying geometrically to
    lr_end if given); returns the loss history."""
    rmax = float(R.max())
    graphs = []
    for a, b in pairs:
        g = make_graph(a["x"], a["v"], a["w"], R, rmax)
        T = targets(a["v"], a["w"], b["v"], b["w"], R, stride, dt, SCALES["a_s"])
        graphs.append((g, target_buffer(T, g.npad)))
    hist = []
    for it in range(iters):
        g, T = graphs[it % len(graphs)]
        loss = model.loss_and_grad(g, T)
        rate = lr if lr_end is None else lr * (lr_end / lr) ** (it / max(1, iters - 1))
        model.adam(rate)
        if it % log_every == 0 or it == iters - 1:
            hist.append((it, loss))
    return hist


def predict(model: MPNN, state, R):
    g = make_graph(state["x"], state["v"], state["w"], R, float(R.max()))
    y = model.forward(g, keep=False)
    return y[:g.n, :OUT].cpu().numpy().astype(np.float64) * SCALES["a_s"]


def evaluate(model: MPNN, pairs, R, dt, g_vec, stride=10):
    """Mean squared error (scaled units) of the network and of the
    gravity-only guess (a = g, alpha = 0) on held-out pairs."""
    e_net, e_base = [], []
    for a, b in pairs:
        T = targets(a["v"], a["w"], b["v"], b["w"], R, stride, dt, 1.0)
        P = predict(model, a, R)
        base = np.zeros_like(T)
        base[:, :3] = g_vec
        e_net.append(np.mean(((P - T) / SCALES["a_s"]) ** 2))
        e_base.append(np.mean(((base - T) / SCALES["a_s"]) ** 2))
    return float(np.mean(e_net)), float(np.mean(e_base))


def advance(state, acc, R, dt, stride):
    """Semi-implicit Euler over `stride` steps with constant predicted
    accelerations (a, R alpha): v_k = v + k a dt, x += sum_k v_k dt."""
    a, al = acc[:, :3], acc[:, 3:] / R[:, None]
    k = stride
    v1 = state["v"] + k * dt * a
    x1 = state["x"] + k * dt * state["v"] + dt * dt * a * (k * (k + 1) / 2.0)
    w1 = state["w"] + k * dt * al
    return dict(x=x1, v=v1, w=w1, q=state["q"])


def max_overlap(x, R, rmax):
    """Largest overlap / radius among neighbours (from the surrogate's graph)."""
    g = make_graph(x, np.zeros_like(x), np.zeros_like(x), R, rmax)
    off, nbr, dst = g.edges_host()
    if len(nbr) == 0:
        return 0.0
    d = np.linalg.norm(x[nbr] - x[dst], axis=1)
    return float(np.max((R[nbr] + R[dst] - d) / np.minimum(R[nbr], R[dst])))


def rollout(model: MPNN, state, R, params, strides, stride=10, overlap_growth=0.02,
            energy_limit=0.5, precision=1):
    """Hybrid run: each stride, the network's accelerations advance the state
    unless the largest overlap grows by more than overlap_growth R_min or the
    kinetic energy changes by more than energy_limit (relative); then the DEM
    takes that stride from the state before it.  Also runs the DEM alone
    alongside and returns the per-stride position error of the hybrid
    (RMS / R_max)."""
    import time
    dt = params["dt"]
    rmax = float(R.max())
    rho = params["rho"]
    m = 4.0 / 3.0 * math.pi * rho * R ** 3

    def ke(s):
        return 0.5 * float(np.sum(m * np.einsum("ij,ij->i", s["v"], s["v"])))

    def dem_stride(s):
        sc = _dem.Scene(params, R, s["x"], s["v"], s["w"], s["q"], precision=precision,
                        **_mesh_kw)
        sc.step(stride)
        out = sc.state()
        sc.close()
        return out

    ref = dict(state)
    cur = dict(state)
    rows = []
    t_net = t_dem = 0.0
    falls = 0
    for k in range(strides):
        t0 = time.perf_counter()
        acc = predict(model, cur, R)
        nxt = advance(cur, acc, R, dt, stride)
        ov0 = max_overlap(cur["x"], R, rmax)
        ov = max_overlap(nxt["x"], R, rmax)
        e0, e1 = ke(cur), ke(nxt)
        t_net += time.perf_counter() - t0
        if ov > ov0 + overlap_growth or abs(e1 - e0) > energy_limit * max(e0, 1e-30):
            t0 = time.perf_counter()
            nxt = dem_stride(cur)
            t_dem += time.perf_counter() - t0
            falls += 1
        cur = nxt
        ref = dem_stride(ref)
        err = float(np.sqrt(np.mean(np.sum((cur["x"] - ref["x"]) ** 2, axis=1)))) / rmax
        rows.append((k + 1, err, ov))
    return {"strides": strides, "fallbacks": falls, "pos_error_rms_over_rmax": rows,
            "net_s": t_net, "dem_fallback_s": t_dem}


_mesh_kw = {}


def experiment(n_scenes=16, n_train=80, n_eval=16, iters=3000, lr=1e-3, drum_n=100_000,
               strides=10, seed=0):
    """Train on hopper-discharge trajectories (the batched workload), evaluate
    on held-out pairs against the gravity-only guess, then run the network on
    a rotating drum with DEM fallback.  Returns a dict of the results."""
    import time
    from . import batch, scenes
    rng = np.random.default_rng(seed)
    ns = [int(n) for n in np.exp(rng.uniform(math.log(800), math.log(3000), n_scenes))]
    mus = [(float(rng.uniform(0.2, 0.8)), float(rng.uniform(0, 0.2)),
            float(rng.uniform(0, 0.2))) for _ in ns]
    b = batch.combine([batch.hopper_scene(n, 700 + k, mus[k]) for k, n in enumerate(ns)])
    dt = b["params"]["dt"]
    t0 = time.perf_counter()
    pairs, R = sample_pairs(b, n_train + n_eval, every=100, settle=3000)
    t_data = time.perf_counter() - t0
    model = MPNN(seed=seed)
    t0 = time.perf_counter()
    hist = train(model, pairs[:n_train], R, dt, iters=iters, lr=lr, lr_end=lr / 10,
                 log_every=max(1, iters // 12))
    t_train = time.perf_counter() - t0
    gv = np.asarray(b["params"]["g"])
    e_net, e_base = evaluate(model, pairs[n_train:], R, dt, gv)
    t_net_mse, t_base_mse = evaluate(model, pairs[:n_train], R, dt, gv)
    # the network on a drum (another geometry), with DEM fallback
    d = scenes.drum_scene(n=drum_n, seed=5, n_theta=64, n_rings=8, nn_dist=2.15e-3, speed=0.02)
    sc = _dem.Scene.from_dict(d, precision=1)
    sc.step(1500)
    st = sc.state()
    # DEM time for one stride of the drum, graph replay (device)
    sc.synchronize()
    t0 = time.perf_counter()
    sc.step(100)
    sc.synchronize()
    dem_stride_ms = (time.perf_counter() - t0) * 1e3 / 10
    sc.close()
    _mesh_kw.clear()
    _mesh_kw.update(verts=d["verts"], tris=d["tris"], tri_radius=d["tri_radius"])
    roll = rollout(model, st, d["R"], d["params"], strides)
    # network time for one stride of the drum: graph + forward
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        predict(model, st, d["R"])
    torch.cuda.synchronize()
    net_stride_ms = (time.perf_counter() - t0) * 1e3 / 5
    return {"train_particles": int(len(R)), "train_pairs": n_train, "eval_pairs": n_eval,
            "iters": iters, "loss_history": hist, "eval_mse_net": e_net,
            "eval_mse_gravity_only": e_base, "train_mse_net": t_net_mse,
            "train_mse_gravity_only": t_base_mse, "data_s": t_data, "train_s": t_train,
            "drum_particles": drum_n, "rollout": roll,
            "net_ms_per_stride": net_stride_ms, "dem_ms_per_stride": dem_stride_ms}


def main():
    import json
    import argparse
    ap = argparse.ArgumentParser(description="train and run the surrogate")
    ap.add_argument("--iters", type=int, default=3000)
    ap.add_argument("--drum-n", type=int, default=100_000)
    ap.add_argument("--strides", type=int, default=10)
    a = ap.parse_args()
    print(json.dumps(experiment(iters=a.iters, drum_n=a.drum_n, strides=a.strides)))


if __name__ == "__main__":
    main()
