"""Learned warm start for the crossbar solve (a throughput pattern on top of the paper's
method, not part of it).

A six-layer dilated CNN maps a crossbar's conductance map and input vector (plus the
node position) to a guess of both layers' node voltages.  It is trained on solves the
method itself produces, and the guess only seeds Newton: ``Solver.solve_from`` rejects
a guess whose KCL residual is not below that of V = 0 (then the linear-circuit start is
used) and always iterates to the requested tolerance, so the network can save work but
never change the answer.

Every arithmetic step runs in the library's kernels (convolutions forward and backward,
leaky ReLU, MSE, Adam, feature and state conversion); PyTorch only provides device
buffers.  Run ``python -m paper_2109_07929_gb300.cnn --help`` to train and evaluate.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import struct
import time

import numpy as np

from . import (PREC_BF16_SPLIT, Solver, _check, _ptr, _stream_ptr, default_params, load)

# (cin, cout, dilation, leaky-ReLU) per layer: 6 layers, 32 channels, receptive field 127
LAYERS = ((4, 32, 1, 1), (32, 32, 2, 1), (32, 32, 4, 1), (32, 32, 8, 1), (32, 32, 16, 1),
          (32, 2, 32, 0))
VSCALE = 0.3      # volts: V_in ~ U[0, 0.3]
BSCALE = 4.0      # bottom-layer voltages are ~4x smaller than the top layer's
NCHAN = 4         # log g, V_in, column position, row position
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                       "warmstart_cnn.bin")
_MAGIC = b"MCACNN01"


class WarmStartCNN:
    def __init__(self, seed=0, device="cuda"):
        import torch
        self.torch = torch
        self.lib = load()
        self.dev = torch.device(device)
        rng = np.random.default_rng(seed)
        self.w, self.b = [], []
        for cin, cout, d, act in LAYERS:
            std = np.sqrt(2.0 / (cin * 9)) if act else 1e-2
            self.w.append(torch.as_tensor(rng.standard_normal((cout, cin, 3, 3)) * std,
                                          dtype=torch.float32, device=self.dev))
            self.b.append(torch.zeros(cout, dtype=torch.float32, device=self.dev))
        self._sync_bf16()
        self.mw = [torch.zeros_like(w) for w in self.w]
        self.vw = [torch.zeros_like(w) for w in self.w]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.step = 0

    def n_params(self):
        return int(sum(w.numel() + b.numel() for w, b in zip(self.w, self.b)))

    def _sync_bf16(self):
        torch = self.torch
        self.wb = [w.to(torch.bfloat16).view(torch.int16).contiguous() for w in self.w]

    # ---- forward / backward through the library kernels -------------------------------
    def forward(self, x, N, H, W, stream=None):
        torch = self.torch
        acts = [x]
        for (cin, cout, d, act), wb, b in zip(LAYERS, self.wb, self.b):
            y = torch.empty(N, cout, H, W, dtype=torch.float32, device=self.dev)
            _check(self.lib.mca_cnn_conv_forward(_ptr(acts[-1]), N, cin, H, W, _ptr(wb), _ptr(b),
                                                 cout, d, act, _ptr(y), _stream_ptr(stream)))
            acts.append(y)
        return acts

    def train_step(self, x, target, N, H, W, lr, stream=None, nchunk=64):
        torch = self.torch
        acts = self.forward(x, N, H, W, stream)
        pred = acts[-1]
        g = torch.empty_like(pred)
        part = torch.empty(256, dtype=torch.float32, device=self.dev)
        loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        _check(self.lib.mca_cnn_mse(_ptr(pred), _ptr(target), pred.numel(), _ptr(g), _ptr(part),
                                    _ptr(loss), _stream_ptr(stream)))
        self.step += 1
        for li in range(len(LAYERS) - 1, -1, -1):
            cin, cout, d, act = LAYERS[li]
            gz = torch.empty_like(acts[li + 1])
            gx = torch.empty_like(acts[li]) if li > 0 else None
            gw = torch.empty_like(self.w[li])
            gb = torch.empty_like(self.b[li])
            pbuf = torch.empty(nchunk * (cout * cin * 9 + cout), dtype=torch.float32,
                               device=self.dev)
            _check(self.lib.mca_cnn_conv_backward(
                _ptr(acts[li]), _ptr(acts[li + 1]), _ptr(g), N, cin, H, W, _ptr(self.wb[li]),
                cout, d, act, _ptr(gz), _ptr(gx), _ptr(gw), _ptr(gb), _ptr(pbuf), nchunk,
                _stream_ptr(stream)))
            for p, gp, m1, m2, pb in ((self.w[li], gw, self.mw[li], self.vw[li], self.wb[li]),
                                      (self.b[li], gb, self.mb[li], self.vb[li], None)):
                _check(self.lib.mca_cnn_adam(_ptr(p), _ptr(pb), _ptr(gp), _ptr(m1), _ptr(m2),
                                             p.numel(), lr, 0.9, 0.999, 1e-8, self.step,
                                             _stream_ptr(stream)))
            g = gx
        return loss

    # ---- guesses ------------------------------------------------------------------------
    def features(self, gmap_dev, vin_dev, m, n, stream=None):
        torch = self.torch
        nv = vin_dev.shape[0]
        x = torch.empty(nv, NCHAN, m, n, dtype=torch.float32, device=self.dev)
        _check(self.lib.mca_cnn_features(_ptr(gmap_dev), _ptr(vin_dev), nv, m, n, VSCALE, NCHAN,
                                         _ptr(x), _stream_ptr(stream)))
        return x

    def targets(self, state_dev, m, n, stream=None):
        torch = self.torch
        nv = state_dev.shape[0]
        y = torch.empty(nv, 2, m, n, dtype=torch.float32, device=self.dev)
        _check(self.lib.mca_cnn_state(None, _ptr(state_dev), nv, m, n, VSCALE, BSCALE, 0, _ptr(y),
                                      _stream_ptr(stream)))
        return y

    def guess(self, gmap_dev, vin_dev, m, n, stream=None):
        """FP64 initial states [V_t ; V_b] (nvec, 2*m*n) for Solver.solve_from."""
        torch = self.torch
        nv = vin_dev.shape[0]
        x = self.features(gmap_dev, vin_dev, m, n, stream)
        y = self.forward(x, nv, m, n, stream)[-1]
        st = torch.empty(nv, 2 * m * n, dtype=torch.float64, device=self.dev)
        _check(self.lib.mca_cnn_state(_ptr(y), _ptr(st), nv, m, n, VSCALE, BSCALE, 1, None,
                                      _stream_ptr(stream)))
        return st

    # ---- weights file: magic, layer count, (cin, cout, d, act) per layer, FP32 w and b --
    def save(self, path=WEIGHTS):
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "wb") as f:
            f.write(_MAGIC)
            f.write(struct.pack("<i", len(LAYERS)))
            for spec in LAYERS:
                f.write(struct.pack("<4i", *spec))
            for w, b in zip(self.w, self.b):
                f.write(w.detach().cpu().numpy().astype("<f4").tobytes())
                f.write(b.detach().cpu().numpy().astype("<f4").tobytes())

    def load(self, path=WEIGHTS):
        torch = self.torch
        with open(path, "rb") as f:
            if f.read(8) != _MAGIC:
                raise ValueError("not a warm-start weights file")
            (nl,) = struct.unpack("<i", f.read(4))
            specs = [tuple(struct.unpack("<4i", f.read(16))) for _ in range(nl)]
            if tuple(specs) != LAYERS:
                raise ValueError("weights file was written for another architecture")
            for li, (cin, cout, d, act) in enumerate(specs):
                w = np.frombuffer(f.read(cout * cin * 9 * 4), dtype="<f4").reshape(cout, cin, 3, 3)
                b = np.frombuffer(f.read(cout * 4), dtype="<f4")
                self.w[li] = torch.as_tensor(w.copy(), device=self.dev)
                self.b[li] = torch.as_tensor(b.copy(), device=self.dev)
        self._sync_bf16()
        return self


# ---- data, training and evaluation --------------------------------------------------------

def _params(p, **kw):
    return default_params(p.rows, p.cols, g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot,
                          g_src=p.g_src, g_term_top_right=p.g_term_top_right,
                          g_term_bot_top=p.g_term_bot_top, g_sense=p.g_sense, b=p.b, **kw)


def make_dataset(count, size=256, seed0=1_000_000, group=64, log=print):
    """`count` crossbars of the small-workload distribution (log-uniform g in [1e-6,1e-4]
    S, 1 S wires, V_in ~ U[0, 0.3]) solved to 1e-10 by the library; returns device
    tensors (features, targets, gmaps, vins)."""
    import torch
    import mca_inputs as mi
    model = WarmStartCNN.__new__(WarmStartCNN)          # feature/target helpers only
    model.torch, model.lib, model.dev = torch, load(), torch.device("cuda")
    X, T, G, V = [], [], [], []
    solver = None
    t0 = time.time()
    for g0 in range(0, count, group):
        k = min(group, count - g0)
        cbs = [mi.make_crossbar(size, size, seed0 + g0 + i) for i in range(k)]
        gm = np.stack([cb.gmap for cb in cbs])
        vin = np.concatenate([cb.vin for cb in cbs])
        if solver is None or solver.n_maps != k:
            if solver is not None:
                solver.close()
            solver = Solver(_params(cbs[0].params, precision=PREC_BF16_SPLIT, newton_rtol=1e-10,
                                    max_batch=k), gm)
        else:
            solver.set_conductances(gm)
        vin_d = torch.as_tensor(vin, device="cuda")
        vt = torch.empty(k, size, size, dtype=torch.float64, device="cuda")
        vb = torch.empty_like(vt)
        io = torch.empty(k, size, dtype=torch.float64, device="cuda")
        solver.solve(vin_d, vt, vb, io, map_index=np.arange(k))
        state = torch.cat([vt.reshape(k, -1), vb.reshape(k, -1)], dim=1).contiguous()
        gm_d = torch.as_tensor(gm, device="cuda")
        for i in range(k):
            X.append(model.features(gm_d[i], vin_d[i:i + 1], size, size))
        T.append(model.targets(state, size, size))
        G.append(gm_d)
        V.append(vin_d)
    if solver is not None:
        solver.close()
    torch.cuda.synchronize()
    log(f"dataset: {count} solves of {size}^2 in {time.time() - t0:.1f} s")
    return torch.cat(X), torch.cat(T), torch.cat(G), torch.cat(V)


def train(model, X, T, epochs=4, batch=32, lr=2e-3, log=print):
    import torch
    N, _, H, W = X.shape
    steps = epochs * ((N + batch - 1) // batch)
    it = 0
    losses = []
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(N, device=X.device, generator=None)
        for s0 in range(0, N, batch):
            idx = perm[s0:s0 + batch]
            xb = X[idx].contiguous()
            tb = T[idx].contiguous()
            lr_t = 1e-4 + 0.5 * (lr - 1e-4) * (1 + np.cos(np.pi * it / max(1, steps)))
            loss = model.train_step(xb, tb, xb.shape[0], H, W, lr_t)
            it += 1
            if it % 50 == 0 or it == steps:
                losses.append(float(loss.item()))
                log(f"epoch {ep} step {it}/{steps} loss {losses[-1]:.3e} "
                    f"({time.time() - t0:.0f} s)")
    torch.cuda.synchronize()
    return losses, time.time() - t0


def evaluate(model, size, count, seed0=2_000_000, log=print):
    """Newton from V = 0 vs from the CNN guess on held-out crossbars of `size`."""
    import torch
    import mca_inputs as mi
    rows = []
    for k in range(count):
        cb = mi.make_crossbar(size, size, seed0 + k)
        p = _params(cb.params, precision=PREC_BF16_SPLIT, newton_rtol=1e-8, max_batch=1)
        with Solver(p, cb.gmap) as s:
            gm_d = torch.as_tensor(cb.gmap, device="cuda")
            vin_d = torch.as_tensor(cb.vin, device="cuda")
            vt = torch.empty(1, size, size, dtype=torch.float64, device="cuda")
            vb = torch.empty_like(vt)
            io = torch.empty(1, size, dtype=torch.float64, device="cuda")
            s.solve(vin_d, vt, vb, io)                      # warm-up (graphs)
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, _, _, st0 = s.solve(vin_d, vt, vb, io)
            torch.cuda.synchronize()
            t_base = time.perf_counter() - t
            ref = torch.cat([vt.reshape(1, -1), vb.reshape(1, -1)], dim=1)
            g = model.guess(gm_d, vin_d, size, size)
            s.solve_from(vin_d, g, vt, vb, io)
            torch.cuda.synchronize()
            t = time.perf_counter()
            g = model.guess(gm_d, vin_d, size, size)
            _, _, _, st1 = s.solve_from(vin_d, g, vt, vb, io)
            torch.cuda.synchronize()
            t_warm = time.perf_counter() - t
            err = float(((g - ref).abs().max() / ref.abs().max()).item())
        rows.append(dict(newton_base=st0[0]["newton_iters"], gmres_base=st0[0]["gmres_iters"],
                         newton_warm=st1[0]["newton_iters"], gmres_warm=st1[0]["gmres_iters"],
                         fallback=st1[0]["fallback"], residual_warm=st1[0]["rel_residual"],
                         guess_max_rel_err=err, t_base_ms=1e3 * t_base,
                         t_warm_ms=1e3 * t_warm))
        log(f"{size}^2 #{k}: {rows[-1]}")
    agg = {key: float(np.mean([r[key] for r in rows])) for key in rows[0]}
    agg["count"] = count
    agg["newton_iters_saved"] = agg["newton_base"] - agg["newton_warm"]
    agg["gmres_iters_saved"] = agg["gmres_base"] - agg["gmres_warm"]
    agg["fallback_rate"] = agg.pop("fallback")
    agg["max_residual_warm"] = float(max(r["residual_warm"] for r in rows))
    return agg


def main():
    ap = argparse.ArgumentParser(description="train / evaluate the warm-start CNN")
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--eval256", type=int, default=8)
    ap.add_argument("--eval512", type=int, default=8)
    ap.add_argument("--eval1024", type=int, default=4)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--report", default=None, help="write the evaluation JSON here")
    ap.add_argument("--eval-only", action="store_true")
    a = ap.parse_args()
    model = WarmStartCNN(seed=0)
    print(f"parameters: {model.n_params()}")
    report = {"parameters": model.n_params(), "layers": LAYERS}
    if not a.eval_only:
        X, T, _, _ = make_dataset(a.samples, a.size)
        losses, ttrain = train(model, X, T, a.epochs, a.batch, a.lr)
        del X, T
        model.save(a.out)
        report.update(train_samples=a.samples, train_size=a.size, epochs=a.epochs,
                      final_loss=losses[-1], train_seconds=ttrain)
    else:
        model.load(a.out)
    report["eval_256_in_distribution"] = evaluate(model, 256, a.eval256)
    report["eval_512"] = evaluate(model, 512, a.eval512)
    report["eval_1024"] = evaluate(model, 1024, a.eval1024)
    print(json.dumps(report))
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
