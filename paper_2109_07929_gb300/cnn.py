"""Learned warm start for the crossbar solve (a throughput pattern on top of the paper's
method, not part of it).

The first Newton step from V = 0 is the linear-circuit solve; what is left after it is
the nonlinear correction V* - V_lin.  A six-layer convolutional network (11 x 11 kernels,
32 channels, dilations 1 .. 32, about 0.52M parameters, BF16 weights with FP32
accumulation) maps a crossbar's conductance map, its input vector and V_lin to that
correction.  It is trained on solves the method itself produces, and its guess
V_lin + correction only seeds Newton: ``Solver.solve_from`` keeps the guess only when its
KCL residual is below that of V_lin (otherwise Newton continues from V_lin) and always
iterates to the requested tolerance, so the network can save work but never change the
answer.

Every arithmetic step runs in the library's kernels (tensor-core convolutions forward,
backward and weight gradient, loss, Adam, the BF16 operand tiles, features, targets and
guesses); PyTorch only provides device buffers.  Run ``python -m paper_2109_07929_gb300.cnn
--help`` to train and evaluate.
"""
from __future__ import annotations

import argparse
import json
import os
import struct
import time

import numpy as np

from . import (PREC_BF16_SPLIT, Solver, _check, _ptr, _stream_ptr, default_params, load,
               residual_noalloc)

# (cin, cout, dilation, leaky-ReLU) per layer; 11 x 11 kernels: receptive field 631 nodes
LAYERS = ((4, 32, 1, 1), (32, 32, 2, 1), (32, 32, 4, 1), (32, 32, 8, 1), (32, 32, 16, 1),
          (32, 2, 32, 0))
KSIZE = 11
C = 32            # channels of the NHWC activation tensors (padded)
VSCALE = 0.3      # volts: V_in ~ U[0, 0.3]
BSCALE = 4.0      # bottom-layer voltages are ~4x smaller than the top layer's
DSCALE = 2000.0   # 1/V: the correction V* - V_lin is a few 1e-4 V
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights",
                       "warmstart_cnn11.bin")
_MAGIC = b"MCACNN02"


def _cout_mma(cout):
    return 16 if cout <= 16 else 32


class WarmStartCNN:
    def __init__(self, seed=0, device="cuda"):
        import torch
        self.torch = torch
        self.lib = load()
        self.dev = torch.device(device)
        rng = np.random.default_rng(seed)
        T = KSIZE * KSIZE
        self.w, self.b, self.wf, self.wb = [], [], [], []
        for cin, cout, d, act in LAYERS:
            std = np.sqrt(2.0 / (cin * T)) if act else 1e-3
            self.w.append(torch.as_tensor(rng.standard_normal((cout, cin, KSIZE, KSIZE)) * std,
                                          dtype=torch.float32, device=self.dev))
            self.b.append(torch.zeros(cout, dtype=torch.float32, device=self.dev))
            self.wf.append(torch.empty(T, _cout_mma(cout), C, dtype=torch.int16, device=self.dev))
            self.wb.append(torch.empty(T, C, C, dtype=torch.int16, device=self.dev))
        self.mw = [torch.zeros_like(w) for w in self.w]
        self.vw = [torch.zeros_like(w) for w in self.w]
        self.mb = [torch.zeros_like(b) for b in self.b]
        self.vb = [torch.zeros_like(b) for b in self.b]
        self.step = 0
        self._scratch = {}
        for li in range(len(LAYERS)):
            self.prep(li)

    def n_params(self):
        return int(sum(w.numel() + b.numel() for w, b in zip(self.w, self.b)))

    def prep(self, li, stream=None):
        """BF16 operand tiles of layer li from its FP32 master weights (library kernel)."""
        cin, cout, d, act = LAYERS[li]
        _check(self.lib.mca_cnn_prep_weights(_ptr(self.w[li]), cout, cin, KSIZE, _cout_mma(cout),
                                             _ptr(self.wf[li]), _ptr(self.wb[li]),
                                             _stream_ptr(stream)))

    def _nhwc(self, N, H, W):
        return self.torch.empty(N, H, W, C, dtype=self.torch.int16, device=self.dev)

    # ---- forward / backward through the library kernels -------------------------------
    def forward(self, x, N, H, W, stream=None):
        """x: NHWC32 BF16 input (N, H, W, 32).  Returns the hidden activations (NHWC32 BF16,
        the input first) and the FP32 prediction (N, H, W, 2)."""
        torch = self.torch
        acts = [x]
        pred = None
        for li, (cin, cout, d, act) in enumerate(LAYERS):
            last = li == len(LAYERS) - 1
            out = None if last else self._nhwc(N, H, W)
            out32 = torch.empty(N, H, W, cout, dtype=torch.float32, device=self.dev) if last else None
            _check(self.lib.mca_cnn_conv(_ptr(acts[-1]), N, H, W, _ptr(self.wf[li]), KSIZE, d,
                                         _cout_mma(cout), cout, _ptr(self.b[li]), act, 0, None,
                                         _ptr(out), _ptr(out32), _stream_ptr(stream)))
            if last:
                pred = out32
            else:
                acts.append(out)
        return acts, pred

    def train_step(self, x, target, N, H, W, lr, stream=None):
        torch = self.torch
        acts, pred = self.forward(x, N, H, W, stream)
        gz = self._nhwc(N, H, W)
        part = torch.empty(256, dtype=torch.float32, device=self.dev)
        loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        _check(self.lib.mca_cnn_loss(_ptr(pred), _ptr(target), N * H * W, _ptr(gz), _ptr(part),
                                     _ptr(loss), _stream_ptr(stream)))
        key = (N, H, W)
        if key not in self._scratch:
            nf = int(self.lib.mca_cnn_wgrad_scratch(N, H, W, KSIZE))
            self._scratch[key] = torch.empty(nf, dtype=torch.float32, device=self.dev)
        scratch = self._scratch[key]
        self.step += 1
        for li in range(len(LAYERS) - 1, -1, -1):
            cin, cout, d, act = LAYERS[li]
            gw = torch.empty_like(self.w[li])
            gb = torch.empty_like(self.b[li])
            _check(self.lib.mca_cnn_conv_wgrad(_ptr(acts[li]), _ptr(gz), N, H, W, KSIZE, d, cin,
                                               cout, _ptr(scratch), _ptr(gw), _ptr(gb),
                                               _stream_ptr(stream)))
            gprev = None
            if li > 0:
                # dL/dz of the layer below: the transposed convolution of gz times the leaky
                # ReLU derivative at that layer's output (this layer's input)
                gprev = self._nhwc(N, H, W)
                _check(self.lib.mca_cnn_conv(_ptr(gz), N, H, W, _ptr(self.wb[li]), KSIZE, d, C,
                                             cin, None, LAYERS[li - 1][3], 1, _ptr(acts[li]),
                                             _ptr(gprev), None, _stream_ptr(stream)))
            for p, g, m1, m2 in ((self.w[li], gw, self.mw[li], self.vw[li]),
                                 (self.b[li], gb, self.mb[li], self.vb[li])):
                _check(self.lib.mca_cnn_adam(_ptr(p), _ptr(g), _ptr(m1), _ptr(m2), p.numel(), lr,
                                             0.9, 0.999, 1e-8, self.step, _stream_ptr(stream)))
            self.prep(li, stream)
            gz = gprev
        return loss

    # ---- inputs, targets, guesses -----------------------------------------------------
    def features(self, gmaps_dev, map_dev, vin_dev, vlt, vlb, m, n, stream=None):
        nv = vin_dev.shape[0]
        x = self._nhwc(nv, m, n)
        _check(self.lib.mca_cnn_features(_ptr(gmaps_dev), _ptr(map_dev), _ptr(vin_dev), _ptr(vlt),
                                         _ptr(vlb), nv, m, n, VSCALE, BSCALE, _ptr(x),
                                         _stream_ptr(stream)))
        return x

    def targets(self, vst, vsb, vlt, vlb, m, n, stream=None):
        torch = self.torch
        nv = vst.shape[0]
        t = torch.empty(nv, m, n, 2, dtype=torch.float32, device=self.dev)
        _check(self.lib.mca_cnn_target(_ptr(vst), _ptr(vsb), _ptr(vlt), _ptr(vlb), nv, m, n,
                                       DSCALE, DSCALE, _ptr(t), _stream_ptr(stream)))
        return t

    def state(self, pred, vlt, vlb, m, n, stream=None):
        """FP64 states [V_t ; V_b] (nvec, 2*m*n): V_lin + the predicted correction, or V_lin
        itself for pred = None."""
        torch = self.torch
        nv = vlt.shape[0]
        st = torch.empty(nv, 2 * m * n, dtype=torch.float64, device=self.dev)
        _check(self.lib.mca_cnn_guess(_ptr(pred), _ptr(vlt), _ptr(vlb), nv, m, n, DSCALE, DSCALE,
                                      _ptr(st), _stream_ptr(stream)))
        return st

    def check(self, stream=None):
        _check(self.lib.mca_cnn_check(_stream_ptr(stream)))

    # ---- weights file: magic, kernel size, layer count, (cin, cout, d, act) per layer, FP32
    # w [cout][cin][K][K] and b per layer
    def save(self, path=WEIGHTS):
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "wb") as f:
            f.write(_MAGIC)
            f.write(struct.pack("<2i", KSIZE, len(LAYERS)))
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
            k, nl = struct.unpack("<2i", f.read(8))
            specs = tuple(tuple(struct.unpack("<4i", f.read(16))) for _ in range(nl))
            if k != KSIZE or specs != LAYERS:
                raise ValueError("weights file was written for another architecture")
            for li, (cin, cout, d, act) in enumerate(specs):
                cnt = cout * cin * KSIZE * KSIZE
                w = np.frombuffer(f.read(cnt * 4), dtype="<f4").reshape(cout, cin, KSIZE, KSIZE)
                b = np.frombuffer(f.read(cout * 4), dtype="<f4")
                self.w[li].copy_(torch.as_tensor(w.copy()))
                self.b[li].copy_(torch.as_tensor(b.copy()))
                self.prep(li)
        return self


# ---- data, training and evaluation --------------------------------------------------------

def _params(p, **kw):
    return default_params(p.rows, p.cols, g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot,
                          g_src=p.g_src, g_term_top_right=p.g_term_top_right,
                          g_term_bot_top=p.g_term_bot_top, g_sense=p.g_sense, b=p.b, **kw)


class SolvePair:
    """Two multi-map handles of one shape: `lin` stops after the first Newton step (V_lin),
    `full` solves to the tolerance (V*, or the warm-started solve)."""

    def __init__(self, size, count, tol=1e-8):
        import torch
        import mca_inputs as mi
        self.torch, self.size, self.count = torch, size, count
        p = mi.make_crossbar(size, size, 0).params
        g = np.full((count, size, size), 1e-5)
        self.lin = Solver(_params(p, precision=PREC_BF16_SPLIT, max_newton=1, max_batch=count), g)
        self.full = Solver(_params(p, precision=PREC_BF16_SPLIT, newton_rtol=tol,
                                   max_batch=count), g)
        dev = torch.device("cuda")
        z = lambda: torch.empty(count, size, size, dtype=torch.float64, device=dev)
        self.vlt, self.vlb, self.vst, self.vsb = z(), z(), z(), z()
        self.io = torch.empty(count, size, dtype=torch.float64, device=dev)
        self.map_host = np.arange(count, dtype=np.int32)
        self.map_dev = torch.as_tensor(self.map_host, device=dev)

    def set(self, cbs):
        torch = self.torch
        gm = np.stack([cb.gmap for cb in cbs])
        self.lin.set_conductances(gm)
        self.full.set_conductances(gm)
        self.gm_dev = torch.as_tensor(gm, device="cuda")
        self.vin_dev = torch.as_tensor(np.concatenate([cb.vin[:1] for cb in cbs]), device="cuda")

    def solve_lin(self):
        return self.lin.solve(self.vin_dev, self.vlt, self.vlb, self.io, map_index=self.map_host,
                              allow_not_converged=True)[3]

    def solve_full(self):
        return self.full.solve(self.vin_dev, self.vst, self.vsb, self.io, map_index=self.map_host)[3]

    def close(self):
        self.lin.close()
        self.full.close()


def train(model, samples=20000, size=256, batch=32, epochs=4, lr=1e-3, seed0=1_000_000,
          log=print, max_seconds=None):
    """Adam on `samples` crossbars of the 32^2 workload's distribution at `size`^2
    (log-uniform g in [1e-6, 1e-4] S, 1 S wires, V_in ~ U[0, 0.3]), generated and solved by
    the library batch by batch (V_lin from the first Newton step, V* to 1e-10).  Stops early
    after max_seconds (the returned step count says how far it got)."""
    import mca_inputs as mi
    torch = model.torch
    pair = SolvePair(size, batch, tol=1e-10)
    steps = epochs * (samples // batch)
    losses, it = [], 0
    t0 = time.time()
    try:
        for ep in range(epochs):
            order = np.random.default_rng(ep).permutation(samples // batch)
            for bi in order:
                if max_seconds is not None and time.time() - t0 > max_seconds:
                    break
                cbs = [mi.make_crossbar(size, size, seed0 + bi * batch + k) for k in range(batch)]
                pair.set(cbs)
                pair.solve_lin()
                pair.solve_full()
                x = model.features(pair.gm_dev, pair.map_dev, pair.vin_dev, pair.vlt, pair.vlb,
                                   size, size)
                t = model.targets(pair.vst, pair.vsb, pair.vlt, pair.vlb, size, size)
                lr_t = 1e-5 + 0.5 * (lr - 1e-5) * (1 + np.cos(np.pi * it / max(1, steps)))
                loss = model.train_step(x, t, batch, size, size, lr_t)
                it += 1
                if it == 1 or it % 50 == 0 or it == steps:
                    losses.append(float(loss.item()))
                    log(f"epoch {ep} step {it}/{steps} loss {losses[-1]:.4e} "
                        f"({time.time() - t0:.0f} s)")
        model.check()
    finally:
        pair.close()
    torch.cuda.synchronize()
    if not losses or losses[-1] != float(loss.item()):
        losses.append(float(loss.item()))
    return losses, time.time() - t0, it


def evaluate(model, size, count, seed0=2_000_000, log=print):
    """Newton from V = 0 against the warm path (first Newton step -> V_lin, the network's
    correction, Newton from the guess with V_lin as the fallback) on held-out crossbars."""
    import mca_inputs as mi
    torch = model.torch
    cbs = [mi.make_crossbar(size, size, seed0 + k) for k in range(count)]
    pair = SolvePair(size, count, tol=1e-8)
    try:
        pair.set(cbs)
        n = size
        # base: Newton from V = 0 (first call builds the CUDA graphs)
        pair.solve_full()
        torch.cuda.synchronize()
        t = time.perf_counter()
        st0 = pair.solve_full()
        torch.cuda.synchronize()
        t_base = time.perf_counter() - t
        # warm path: V_lin, network, Newton from the guess (a first round warms it up)
        res = None
        for rep in range(2):
            torch.cuda.synchronize()
            t = time.perf_counter()
            st1 = pair.solve_lin()
            torch.cuda.synchronize()
            t_lin = time.perf_counter() - t
            t = time.perf_counter()
            x = model.features(pair.gm_dev, pair.map_dev, pair.vin_dev, pair.vlt, pair.vlb, n, n)
            _, pred = model.forward(x, count, n, n)
            guess = model.state(pred, pair.vlt, pair.vlb, n, n)
            vlin = model.state(None, pair.vlt, pair.vlb, n, n)
            torch.cuda.synchronize()
            t_cnn = time.perf_counter() - t
            t = time.perf_counter()
            _, _, _, st2 = pair.full.solve_from(pair.vin_dev, guess, pair.vst, pair.vsb, pair.io,
                                                map_index=pair.map_host, fallback=vlin)
            torch.cuda.synchronize()
            t_from = time.perf_counter() - t
            res = (st1, st2, t_lin, t_cnn, t_from, guess, vlin)
        st1, st2, t_lin, t_cnn, t_from, guess, vlin = res
        # KCL residuals of the guess and of V_lin (the library's FP64 residual kernel)
        F = torch.empty(1, 2 * n * n, dtype=torch.float64, device="cuda")
        D = torch.empty(1, n * n, dtype=torch.float64, device="cuda")
        fn = torch.empty(2, dtype=torch.float64, device="cuda")
        prm = _params(cbs[0].params)
        ratio = []
        for k in range(count):
            for j, st in enumerate((guess, vlin)):
                residual_noalloc(prm, pair.gm_dev[k], st[k:k + 1], pair.vin_dev[k:k + 1], F, D,
                                 fn[j:j + 1])
            f = fn.cpu().numpy()
            ratio.append(float(f[0] / f[1]))
    finally:
        pair.close()
    model.check()
    out = {
        "size": size, "count": count,
        "newton_base": float(np.mean([s["newton_iters"] for s in st0])),
        "gmres_base": float(np.mean([s["gmres_iters"] for s in st0])),
        # warm path: the first Newton step plus the steps from the accepted start
        "newton_warm": float(np.mean([1 + s["newton_iters"] for s in st2])),
        "gmres_warm": float(np.mean([a["gmres_iters"] + b["gmres_iters"]
                                     for a, b in zip(st1, st2)])),
        "fallback_rate": float(np.mean([s["fallback"] for s in st2])),
        "residual_ratio_guess_over_vlin": {"mean": float(np.mean(ratio)), "min": min(ratio),
                                           "max": max(ratio)},
        "max_residual_base": float(max(s["rel_residual"] for s in st0)),
        "max_residual_warm": float(max(s["rel_residual"] for s in st2)),
        "ms_per_solve_base": 1e3 * t_base / count,
        "ms_per_solve_warm": 1e3 * (t_lin + t_cnn + t_from) / count,
        "ms_per_solve_network": 1e3 * t_cnn / count,
    }
    out["newton_iters_saved"] = out["newton_base"] - out["newton_warm"]
    out["gmres_iters_saved"] = out["gmres_base"] - out["gmres_warm"]
    log(json.dumps(out))
    return out


def main():
    ap = argparse.ArgumentParser(description="train / evaluate the warm-start network")
    ap.add_argument("--samples", type=int, default=20000)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval256", type=int, default=8)
    ap.add_argument("--eval512", type=int, default=8)
    ap.add_argument("--eval1024", type=int, default=4)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--report", default=None, help="write the evaluation JSON here")
    ap.add_argument("--eval-only", action="store_true")
    ap.add_argument("--max-minutes", type=float, default=None, help="training time budget")
    a = ap.parse_args()
    model = WarmStartCNN(seed=0)
    print(f"parameters: {model.n_params()}", flush=True)
    report = {"parameters": model.n_params(), "layers": LAYERS, "kernel": KSIZE}
    if not a.eval_only:
        losses, ttrain, nsteps = train(model, a.samples, a.size, a.batch, a.epochs, a.lr,
                                       max_seconds=None if a.max_minutes is None
                                       else 60 * a.max_minutes)
        model.save(a.out)
        report.update(train_samples=a.samples, train_size=a.size, epochs=a.epochs,
                      batch=a.batch, steps=nsteps, loss_first=losses[0], loss_final=losses[-1],
                      losses=losses, train_seconds=ttrain)
    else:
        model.load(a.out)
    report["eval_256_in_distribution"] = evaluate(model, 256, a.eval256)
    report["eval_512"] = evaluate(model, 512, a.eval512)
    report["eval_1024"] = evaluate(model, 1024, a.eval1024)
    print(json.dumps(report), flush=True)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
