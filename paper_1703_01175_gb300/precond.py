"""Learned preconditioner: a 3-D convolutional network on the voxel grid that
maps a residual to a correction (include/h2nn.h), its training on pairs from
the method's own GMRES solves, and its use as the right preconditioner of
flexible GMRES (h2_set_preconditioner / h2_gmres with precond = 1).

Every arithmetic step runs in the library's kernels; this module allocates
device buffers (torch tensors as plain device memory), sequences the kernel
calls and keeps the training state.

Network (defaults): 6 convolution layers 3x3x3, channels 8 -> 32 -> 32 -> 32 ->
32 -> 32 -> 8, ReLU between layers. Input channels: Re/Im of the three field
components of the residual (scaled to unit RMS) and chi = eps_r - 1 of the
voxel; output channels 0..5: Re/Im of the correction (same scaling).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import h2 as h2py

LAYERS = [(8, 32, 1), (32, 32, 1), (32, 32, 1), (32, 32, 1), (32, 32, 1), (32, 8, 0)]
_vp = ctypes.c_void_p


def _nnlib():
    L = h2py.lib()
    if getattr(L, "_nn_ready", False):
        return L
    i32, i64, f32, fp, dp = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p
    sig = {
        "h2nn_conv3d_fwd": [fp, fp, fp, fp, fp, i32, i32, i32, i32, i32, i32, i32, fp],
        "h2nn_flip_weights": [fp, fp, i32, i32, fp],
        "h2nn_conv3d_bwd_weight": [fp, fp, fp, fp, i32, i32, i32, i32, i32, i32, i32, fp],
        "h2nn_relu_bwd": [fp, fp, fp, i64, fp],
        "h2nn_f32_to_bf16": [fp, fp, i64, fp],
        "h2nn_mse": [fp, fp, fp, fp, i32, i64, i32, i32, fp],
        "h2nn_adam": [fp, fp, fp, fp, fp, i64, f32, f32, f32, f32, i32, fp],
        "h2nn_pack": [fp, i64, fp, fp, fp, fp, i32, i32, i64, fp],
        "h2nn_unpack": [fp, i32, fp, fp, fp, i64, i32, i32, i64, fp],
        "h2_set_preconditioner": [fp, i32, i32, i32, fp, fp, i32, fp, fp, fp],
        "h2nn_device_status": [],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.restype = ctypes.c_int
        f.argtypes = args
    L._nn_ready = True
    return L


def _p(t):
    return None if t is None else _vp(t.data_ptr())


def _call(name, *args):
    st = getattr(_nnlib(), name)(*args)
    if st != 0:
        L = h2py.lib()
        raise h2py.H2Error(st, name, L.h2_last_error().decode())


class ConvNet:
    """Device-resident network state (FP32 master weights, bf16 copies, Adam moments)."""

    def __init__(self, dims, batch, device="cuda", layers=LAYERS, seed=17):
        import torch
        self.torch = torch
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.B = int(batch)
        self.layers = list(layers)
        self.dev = torch.device(device)
        self.W, self.Wb, self.Wt, self.b = [], [], [], []
        self.gW, self.gb, self.mW, self.vW, self.mb, self.vb = [], [], [], [], [], []
        import synth
        for li, (ci, co, relu) in enumerate(self.layers):
            fan_in = 27 * ci
            bound = math.sqrt(6.0 / fan_in) * (0.1 if li == len(self.layers) - 1 else 1.0)
            u = synth.uniform(seed, co * 27 * ci, stream=100 + li).reshape(co, 27, ci)
            w = torch.tensor((2.0 * u - 1.0) * bound, dtype=torch.float32, device=self.dev)
            self.W.append(w.contiguous())
            self.b.append(torch.zeros(co, dtype=torch.float32, device=self.dev))
            self.Wb.append(w.to(torch.bfloat16).contiguous())
            self.Wt.append(torch.empty((ci, 27, co), dtype=torch.bfloat16, device=self.dev))
            for lst, shape in ((self.gW, w.shape), (self.mW, w.shape), (self.vW, w.shape)):
                lst.append(torch.zeros(shape, dtype=torch.float32, device=self.dev))
            for lst in (self.gb, self.mb, self.vb):
                lst.append(torch.zeros(co, dtype=torch.float32, device=self.dev))
        self.step_count = 0
        self._alloc(self.B)

    def _alloc(self, B):
        t = self.torch
        self.acts = [t.empty((B, self.V, ci), dtype=t.bfloat16, device=self.dev) for ci, _, _ in self.layers]
        self.out = t.empty((B, self.V, self.layers[-1][1]), dtype=t.float32, device=self.dev)
        cmax = max(max(ci, co) for ci, co, _ in self.layers)
        self.g1 = t.empty((B, self.V, cmax), dtype=t.float32, device=self.dev)
        self.g2 = t.empty((B, self.V, cmax), dtype=t.float32, device=self.dev)
        self.gbf = t.empty((B, self.V, cmax), dtype=t.bfloat16, device=self.dev)
        self.loss_parts = t.zeros(2 * B, dtype=t.float32, device=self.dev)
        self.B = B

    def stream(self):
        return _vp(self.torch.cuda.current_stream(self.dev).cuda_stream)

    def forward(self, x_bf16):
        """x: bf16 [B][V][8] -> self.out f32 [B][V][8]; keeps the layer inputs."""
        Dx, Dy, Dz = self.dims
        st = self.stream()
        self.acts[0].copy_(x_bf16)
        for li, (ci, co, relu) in enumerate(self.layers):
            last = li == len(self.layers) - 1
            _call("h2nn_conv3d_fwd", _p(self.acts[li]), _p(self.Wb[li]), _p(self.b[li]),
                  None if last else _p(self.acts[li + 1]), _p(self.out) if last else None,
                  self.B, Dx, Dy, Dz, ci, co, relu, st)
        return self.out

    def backward(self, grad_out):
        """Gradients of all parameters from d loss / d out (f32 [B][V][Cout_last])."""
        Dx, Dy, Dz = self.dims
        st = self.stream()
        B, V = self.B, self.V
        g = grad_out
        for li in range(len(self.layers) - 1, -1, -1):
            ci, co, relu = self.layers[li]
            gv = g.reshape(-1)[:B * V * co]
            if relu:
                # the layer's output is the next layer's input
                _call("h2nn_relu_bwd", _p(gv), _p(self.acts[li + 1]), _p(gv), B * V * co, st)
            _call("h2nn_conv3d_bwd_weight", _p(gv), _p(self.acts[li]), _p(self.gW[li]), _p(self.gb[li]),
                  B, Dx, Dy, Dz, ci, co, 0, st)
            if li == 0:
                break
            _call("h2nn_flip_weights", _p(self.Wb[li]), _p(self.Wt[li]), ci, co, st)
            _call("h2nn_f32_to_bf16", _p(gv), _p(self.gbf), B * V * co, st)
            nxt = self.g1 if g is self.g2 else self.g2
            _call("h2nn_conv3d_fwd", _p(self.gbf), _p(self.Wt[li]), None, None, _p(nxt),
                  B, Dx, Dy, Dz, co, ci, 0, st)
            g = nxt

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step_count += 1
        st = self.stream()
        for li in range(len(self.layers)):
            _call("h2nn_adam", _p(self.W[li]), _p(self.gW[li]), _p(self.mW[li]), _p(self.vW[li]), _p(self.Wb[li]),
                  self.W[li].numel(), lr, beta1, beta2, eps, self.step_count, st)
            _call("h2nn_adam", _p(self.b[li]), _p(self.gb[li]), _p(self.mb[li]), _p(self.vb[li]), None,
                  self.b[li].numel(), lr, beta1, beta2, eps, self.step_count, st)

    def loss_and_grad(self, target):
        """Relative squared error against target f32 [B][V][C]; gradient into g1."""
        C = self.layers[-1][1]
        g = self.g1.reshape(-1)[:self.B * self.V * C].view(self.B, self.V, C)
        _call("h2nn_mse", _p(self.out), _p(target), _p(g), _p(self.loss_parts), self.B, self.V, C, 6,
              self.stream())
        return g

    def parameters_numpy(self):
        return {"layers": np.array(self.layers, dtype=np.int32),
                **{f"W{i}": w.cpu().numpy() for i, w in enumerate(self.W)},
                **{f"b{i}": b.cpu().numpy() for i, b in enumerate(self.b)}}

    def load_numpy(self, d):
        for i in range(len(self.layers)):
            self.W[i].copy_(self.torch.from_numpy(np.asarray(d[f"W{i}"], dtype=np.float32)))
            self.b[i].copy_(self.torch.from_numpy(np.asarray(d[f"b{i}"], dtype=np.float32)))
            self.Wb[i].copy_(self.W[i].to(self.torch.bfloat16))

    def n_params(self):
        return sum(w.numel() for w in self.W) + sum(b.numel() for b in self.b)


class GridMap:
    """Tree order <-> voxel grid of a full Dx x Dy x Dz grid workload."""

    def __init__(self, dims, perm, eps_r, device="cuda"):
        import torch
        self.dims = tuple(int(d) for d in dims)
        self.nv = int(len(perm))
        self.V = int(np.prod(self.dims))
        assert self.nv == self.V, "the preconditioner needs every grid voxel as an unknown"
        self.grid_of = torch.tensor(np.asarray(perm, dtype=np.int32), device=device)  # tree pos -> grid index
        self.aux = torch.tensor((np.real(eps_r) - 1.0).astype(np.float32), device=device)

    def pack(self, vecs, scale, out_bf16, stream):
        """vecs: c128 [B][3 nv] (row per sample) -> out bf16 [B][V][8]."""
        B = vecs.shape[0]
        _call("h2nn_pack", _p(vecs), vecs.stride(0), _p(self.grid_of), _p(self.aux), _p(scale), _p(out_bf16),
              B, self.nv, self.V, stream)

    def unpack(self, chan_f32, scale, vecs, stream):
        B = vecs.shape[0]
        _call("h2nn_unpack", _p(chan_f32), chan_f32.shape[-1], _p(self.grid_of), _p(scale), _p(vecs),
              vecs.stride(0), B, self.nv, self.V, stream)


def collect_pairs(A, gm: GridMap, rhs_list, restart=10, tol=1e-6, maxit=4000):
    """Residual -> correction pairs from converged restarted GMRES solves.

    For each right-hand side b: run GMRES(restart) from 0, one cycle per call,
    keeping every restart iterate x_k; continue to a converged x*; the pairs
    are (r_k, e_k) = (b - A x_k, x* - x_k), with r_k from the FP64-accumulated
    product. Returns c128 tensors R, E of shape [P, n] on the device."""
    import torch
    R, E = [], []
    n = A.n
    for b in rhs_list:
        bt = torch.as_tensor(b, dtype=torch.complex128, device="cuda")
        x = torch.zeros_like(bt)
        iters = []
        total = 0
        while total < maxit:
            x, info = A.gmres(bt, x=x, tol=tol, restart=restart, maxit=restart, refine=True, x0_given=True)
            total += max(1, info[0]["iterations"])
            iters.append(x.clone())
            if info[0]["status"] == 0:
                break
        xs = iters[-1]
        for xk in iters[:-1]:
            r = bt - A.matvec(xk, prec="fp64acc")
            R.append(r)
            E.append(xs - xk)
    if not R:
        return None, None
    return torch.stack(R), torch.stack(E)


def collect_pairs_batched(A, B, restart=10, tol=1e-6, maxit=4000, pairs_per_rhs=50, prec="splitbf16",
                          arnoldi="fp32", reorth_eta=0.1):
    """Residual -> correction pairs from the method's own converged solves,
    all right-hand sides in lockstep: batched GMRES(restart) from 0, one cycle
    per call, keeping every restart iterate x_k of every right-hand side;
    once b has converged to x*, up to `pairs_per_rhs` evenly spaced iterates
    give the pairs (r_k, e_k) = (b - A x_k, x* - x_k), r_k from the
    double-float-accumulated product. B: c128 (n, R) column-major on the
    device. Returns c128 tensors R, E of shape [P, n] and the solve record."""
    import torch
    n, nr = B.shape
    X = torch.zeros_like(B)
    iters = [[] for _ in range(nr)]
    done = [False] * nr
    total = 0
    while total < maxit and not all(done):
        X, info = A.gmres_batched(B, X=X, tol=tol, restart=restart, maxit=restart, refine=True, x0_given=True,
                                  prec=prec, arnoldi=arnoldi, reorth_eta=reorth_eta, check=False)
        total += restart
        for r in range(nr):
            if done[r]:
                continue
            iters[r].append(X[:, r].clone())
            if info[r]["status"] == 0:
                done[r] = True
    R, E = [], []
    for r in range(nr):
        if not done[r] or len(iters[r]) < 2:
            continue
        xs, cand = iters[r][-1], iters[r][:-1]
        pick = np.unique(np.linspace(0, len(cand) - 1, min(pairs_per_rhs, len(cand))).round().astype(int))
        bcol = B[:, r].contiguous()
        for k in pick:
            xk = cand[k]
            R.append(bcol - A.matvec(xk.contiguous(), prec="dfacc"))
            E.append(xs - xk)
    record = {"rhs": nr, "converged": int(sum(done)), "steps": total, "restart": restart, "tol": tol}
    if not R:
        return None, None, record
    return torch.stack(R), torch.stack(E), record


def probe_pairs(A, count, seed=7, batch=32):
    """Probe pairs through the method's own product: e random (real and
    imaginary parts uniform in [-1, 1)), r = A e with the FP64-accumulated
    product. They sample the inverse in every direction, whereas restart
    residuals concentrate on the slowly converging modes."""
    import torch
    import synth
    R, E = [], []
    n = A.n
    done = 0
    while done < count:
        k = min(batch, count - done)
        e = torch.from_numpy(np.ascontiguousarray(synth.random_complex(n, seed, stream=300 + done // batch,
                                                                       cols=k).T)).cuda()
        for j in range(k):
            R.append(A.matvec(e[j].contiguous(), prec="fp64acc"))
            E.append(e[j].contiguous())
        done += k
    return torch.stack(R), torch.stack(E)


def train(net: ConvNet, gm: GridMap, R, E, epochs=20, lr=2e-3, seed=3, log=None):
    """Fit net(r_hat) ~ e_hat - r_hat with r_hat = s r, e_hat = s e,
    s = sqrt(n)/|r| per pair: the network learns the correction beyond the
    identity, so that M(r) = r + net(r) ~ A^{-1} r."""
    import torch
    P, n = R.shape
    st = net.stream()
    scale = (math.sqrt(n) / torch.linalg.vector_norm(R, dim=1)).to(torch.float64).contiguous()
    Xb = torch.empty((net.B, net.V, 8), dtype=torch.bfloat16, device=net.dev)
    T = torch.zeros((net.B, net.V, 8), dtype=torch.float32, device=net.dev)
    Tc = torch.zeros((net.B, net.V, 8), dtype=torch.bfloat16, device=net.dev)
    import synth
    history = []
    steps_per_epoch = max(1, P // net.B)
    total = epochs * steps_per_epoch
    step = 0
    for ep in range(epochs):
        order = np.argsort(synth.uniform(seed, P, stream=200 + ep))
        ep_loss = []
        for s in range(steps_per_epoch):
            idx = torch.as_tensor(order[s * net.B:(s + 1) * net.B], device=net.dev)
            if len(idx) < net.B:
                break
            sc = scale[idx].contiguous()
            gm.pack(R[idx].contiguous(), sc, Xb, st)
            gm.pack((E[idx] - R[idx]).contiguous(), sc, Tc, st)
            T.copy_(Tc.float())
            T[..., 6:] = 0.0
            net.forward(Xb)
            g = net.loss_and_grad(T)
            net.backward(g)
            cur_lr = lr * 0.5 * (1 + math.cos(math.pi * step / total))
            net.adam(cur_lr)
            ep_loss.append(net.loss_parts[:net.B].mean())
            step += 1
        mean_loss = float(torch.stack(ep_loss).mean()) if ep_loss else float("nan")
        history.append(mean_loss)
        if log:
            log(f"epoch {ep}: relative loss {mean_loss:.4f}")
    return history


def load_into(A, layers, W, b, gm: GridMap):
    """Copy a network (lists of f32 numpy weights [Cout][27][Cin] and biases)
    into the handle as its flexible-GMRES preconditioner."""
    import torch
    spec = np.array(layers, dtype=np.int32).reshape(-1)
    wb = np.concatenate([torch.from_numpy(np.ascontiguousarray(w, dtype=np.float32)).to(torch.bfloat16)
                         .view(torch.int16).numpy().reshape(-1) for w in W]).astype(np.int16)
    bb = np.concatenate([np.asarray(x, dtype=np.float32).reshape(-1) for x in b]).astype(np.float32)
    grid_of = gm.grid_of.cpu().numpy().astype(np.int32)
    aux = gm.aux.cpu().numpy().astype(np.float32)
    Dx, Dy, Dz = gm.dims
    _call("h2_set_preconditioner", A.handle, Dx, Dy, Dz, grid_of.ctypes.data, aux.ctypes.data, len(layers),
          spec.ctypes.data, wb.ctypes.data, bb.ctypes.data)


def load_net(A, net: ConvNet, gm: GridMap):
    load_into(A, net.layers, [w.cpu().numpy() for w in net.W], [x.cpu().numpy() for x in net.b], gm)


def identity_layers():
    """A one-layer network with zero output: M(v) = v + 0."""
    w = np.zeros((8, 27, 8), dtype=np.float32)
    return [(8, 8, 0)], [w], [np.zeros(8, dtype=np.float32)]


def transpose_arrays(a):
    """H^2 arrays of A^T from those of A = near + sum U^t S^{t,s} W^{sT}:
    row and column bases exchange (U <-> W), couplings and near blocks are
    transposed and move to the mirrored block position (the partition is
    symmetric)."""
    nc = len(a.size)

    def blk(flat, off, r, c):
        return np.asarray(flat[off:off + r * c]).reshape(c, r).T

    leaves = [t for t in range(nc) if a.child[2 * t] < 0]
    parent = np.full(nc, -1)
    for t in range(nc):
        if a.child[2 * t] >= 0:
            parent[a.child[2 * t]] = t
            parent[a.child[2 * t + 1]] = t
    rank, size = a.rank, a.size
    U = {t: blk(a.U, a.U_off[t], size[t], rank[t]) for t in leaves}
    W = U if a.W is None else {t: blk(a.W, a.W_off[t], size[t], rank[t]) for t in leaves}
    T = {t: blk(a.T, a.T_off[t], rank[t], rank[parent[t]]) for t in range(1, nc) if rank[t] and rank[parent[t]]}
    S, Z = {}, {}
    for t in range(nc):
        for j in range(a.adm_ptr[t], a.adm_ptr[t + 1]):
            s = int(a.adm_col[j])
            S[(s, t)] = blk(a.S, a.S_off[j], rank[t], rank[s]).T
        for j in range(a.near_ptr[t], a.near_ptr[t + 1]):
            s = int(a.near_col[j])
            Z[(s, t)] = blk(a.Z, a.Z_off[j], size[t], size[s]).T
    return h2py.arrays_from_blocks(a.n, a.level_ptr, a.child, a.begin, a.size, a.rank, W, U, T, S, Z,
                                   dtype=a.U.dtype)


def train_residual(net: ConvNet, gm: GridMap, A, At, R, epochs=20, lr=2e-3, seed=3, log=None):
    """Fit the preconditioner in residual space: minimise, over the training
    residuals r, ||A M(r) - r||^2 / ||r||^2 with M(r) = r + N(s r) / s,
    s = sqrt(n) / ||r|| (right approximate inverse). The gradient with respect
    to M(r) is 2 A^H (A M(r) - r) / ||r||^2, formed with the transposed
    operator At: A^H y = conj(At conj(y)). Products are batched FP32 H^2
    products; the network runs on the library's convolution kernels."""
    import torch
    import synth
    P_, n = R.shape
    st = net.stream()
    B = net.B
    rnorm = torch.linalg.vector_norm(R, dim=1)
    scale = (math.sqrt(n) / rnorm).to(torch.float64).contiguous()
    inv_scale = (1.0 / scale).contiguous()
    Xb = torch.empty((B, net.V, 8), dtype=torch.bfloat16, device=net.dev)
    Z = torch.empty((B, n), dtype=torch.complex128, device=net.dev)
    Gb = torch.empty((B, net.V, 8), dtype=torch.bfloat16, device=net.dev)
    steps_per_epoch = max(1, P_ // B)
    total = epochs * steps_per_epoch
    step = 0
    history = []
    for ep in range(epochs):
        order = np.argsort(synth.uniform(seed, P_, stream=400 + ep))
        ep_loss = []
        for sidx in range(steps_per_epoch):
            idx = torch.as_tensor(order[sidx * B:(sidx + 1) * B], device=net.dev)
            if len(idx) < B:
                break
            r = R[idx].contiguous()
            sc, isc = scale[idx].contiguous(), inv_scale[idx].contiguous()
            gm.pack(r, sc, Xb, st)
            out = net.forward(Xb)
            gm.unpack(out, isc, Z, st)            # Z = N(s r) / s
            Z += r                                 # M(r)
            Zc = Z.to(torch.complex64).contiguous().T            # (n, B) column-major view
            AZ = A.matvec(Zc).to(torch.complex128)               # (n, B)
            D = AZ - r.T                                          # residual of the preconditioned map
            rn2 = (rnorm[idx] ** 2)
            loss = (torch.linalg.vector_norm(D, dim=0) ** 2 / rn2).mean()
            Dc = D.conj().to(torch.complex64).T.contiguous().T   # conj(D), (n, B) column-major
            G = At.matvec(Dc).to(torch.complex128).conj()         # A^H D
            G = G * (2.0 / (rn2 * B))                             # d loss / d M(r), per column
            # d loss / d out = (d loss / d Z) / s ; pack expects rows per sample
            gm.pack(G.T.contiguous(), isc, Gb, st)
            g = net.g1.reshape(-1)[:B * net.V * 8].view(B, net.V, 8)
            g.copy_(Gb.float())
            g[..., 6:] = 0.0
            net.backward(g)
            cur_lr = lr * 0.5 * (1 + math.cos(math.pi * step / total))
            net.adam(cur_lr)
            ep_loss.append(loss)
            step += 1
        mean_loss = float(torch.stack(ep_loss).mean()) if ep_loss else float("nan")
        history.append(mean_loss)
        if log:
            log(f"epoch {ep}: residual-space loss {mean_loss:.4f}")
    return history
