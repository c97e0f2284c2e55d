"""Learned starting points for the batched fitter.

A multilayer perceptron 256 -> 512 -> 512 -> 11 (GELU; output padded to 16)
maps the 2048-bin histogram of 3 Gaussian peaks + linear background,
rebinned to 256 bins and normalised by its maximum, to starting parameters.
Weights and activations are BF16 with FP32 accumulation; training (forward,
backward, MSE loss, AdamW with FP32 master weights) and inference run in the
kernels of libcg (cg_gemm_bf16 on the tensor cores, cg_rebin_normalize,
cg_mse_loss, cg_colsum, cg_adamw, cg_decode_start).  Targets are the
converged fits of the plain method (the BFGS fitter) on method-generated
histograms.  A learned start is judged by the plain fit (production_fit):
where its fit does not converge, the histogram is fitted again from the
plain heuristic start and the lower minimum is kept.  The paper has no
network; this is the learned-start extension of the batched fitter.
"""
import math

import numpy as np
import torch

from . import cg, synth
from .fit import BatchFitter, HistBatch, TileMap

N_IN, N_HID, N_OUT, N_PAD = 256, 512, 11, 16
FACTOR = 8
N_BINS = 2048
K_PEAKS = 3
FIT_MAP = TileMap(warp_max_bins=4096, cta_max_bins=1 << 30, cta_threads=256, cluster_size=1)
FIT_PRECISION = cg.PREC_DF64   # objective evaluations of the fits on the FP32 pipe (double-float)


def _p(t):
    return cg._ptr(t)


def _s():
    return cg._stream()


def rebin(y_flat, H):
    """bf16 [H, 256] network input and the per-histogram scale (max rebinned count)."""
    x = torch.empty((H, N_IN), dtype=torch.bfloat16, device=y_flat.device)
    scale = torch.empty(H, dtype=torch.float32, device=y_flat.device)
    cg._check(cg.lib().cg_rebin_normalize(_p(y_flat), H, N_BINS, FACTOR, _p(x), _p(scale), _s()),
              "cg_rebin_normalize")
    return x, scale


def heuristic_start(y_flat, H):
    th = torch.empty((H, 3 * K_PEAKS + 2), dtype=torch.float64, device=y_flat.device)
    cg._check(cg.lib().cg_heuristic_start(_p(y_flat), H, N_BINS, FACTOR, 0.0, 1.0, K_PEAKS, _p(th), _s()),
              "cg_heuristic_start")
    return th


REFINE_SWEEPS, REFINE_HALF_WIDTH = 2, 2.5


def refine_start(y_flat, H, theta, sweeps=REFINE_SWEEPS, half_width=REFINE_HALF_WIDTH):
    """Starting parameters sharpened on the full-resolution histogram
    (cg_refine_start: per peak, moments of the counts in a window of
    +-half_width widths less the background and the other peaks)."""
    out = torch.empty_like(theta)
    cg._check(cg.lib().cg_refine_start(_p(y_flat), H, N_BINS, 0.0, 1.0, K_PEAKS, _p(theta.contiguous()), _p(out),
                                       int(sweeps), float(half_width), _s()), "cg_refine_start")
    return out


def canonical(theta):
    """Peaks sorted by mu with positive widths (the fit is symmetric in s and
    in the order of the peaks)."""
    th = theta.clone()
    K = K_PEAKS
    pk = th[:, :3 * K].view(-1, K, 3).clone()
    pk[:, :, 2] = pk[:, :, 2].abs()
    order = torch.argsort(pk[:, :, 1], dim=1)
    pk = torch.gather(pk, 1, order[:, :, None].expand(-1, -1, 3))
    th[:, :3 * K] = pk.reshape(-1, 3 * K)
    return th


# Loss weights per encoded target (A, mu, log s per peak; b0, b1): the
# positions and widths decide where a fit converges.
TARGET_WEIGHTS = [1.0, 3.0, 2.0] * K_PEAKS + [1.0, 1.0]


def encode_targets(theta, scale):
    """Fit parameters [H, 11] -> network targets before z-scoring."""
    theta = canonical(theta)
    f = (FACTOR / scale.double())[:, None]
    t = theta.clone()
    for k in range(K_PEAKS):
        t[:, 3 * k] = theta[:, 3 * k] * f[:, 0]
        t[:, 3 * k + 2] = torch.log(theta[:, 3 * k + 2].abs())
    t[:, 9] = theta[:, 9] * f[:, 0]
    t[:, 10] = theta[:, 10] * f[:, 0]
    return t


class MLP:
    """Parameters, optimiser state and activation buffers of the network."""

    def __init__(self, seed=0, device="cuda"):
        g = torch.Generator().manual_seed(seed)

        def he(o, i, gain=1.0):
            return (torch.randn(o, i, generator=g, dtype=torch.float32) * math.sqrt(2.0 / i) * gain).to(device)

        self.W = [he(N_HID, N_IN), he(N_HID, N_HID), he(N_PAD, N_HID, 0.1)]
        self.W[2][N_OUT:] = 0.0
        self.b = [torch.zeros(N_HID, device=device), torch.zeros(N_HID, device=device),
                  torch.zeros(N_PAD, device=device)]
        self.Wb = [torch.empty(w.shape, dtype=torch.bfloat16, device=device) for w in self.W]
        for w, wb in zip(self.W, self.Wb):
            cg._check(cg.lib().cg_to_bf16(_p(w), w.numel(), _p(wb), _s()), "cg_to_bf16")
        self.params = self.W + self.b
        self.m = [torch.zeros_like(p) for p in self.params]
        self.v = [torch.zeros_like(p) for p in self.params]
        self.grads = [torch.zeros_like(p) for p in self.params]
        self.step = 0
        self.t_mean = torch.zeros(N_OUT, device=device)
        self.t_std = torch.ones(N_OUT, device=device)
        self._buf = {}
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)

    def _bufs(self, B):
        b = self._buf.get(B)
        if b is None:
            dev = self.W[0].device
            f32 = dict(dtype=torch.float32, device=dev)
            b16 = dict(dtype=torch.bfloat16, device=dev)
            b = dict(Z1=torch.empty((B, N_HID), **f32), H1=torch.empty((B, N_HID), **b16),
                     Z2=torch.empty((B, N_HID), **f32), H2=torch.empty((B, N_HID), **b16),
                     Y=torch.empty((B, N_PAD), **f32), dYf=torch.empty((B, N_PAD), **f32),
                     dYb=torch.empty((B, N_PAD), **b16), dZf=torch.empty((B, N_HID), **f32),
                     dZb=torch.empty((B, N_HID), **b16), dZ1f=torch.empty((B, N_HID), **f32),
                     dZ1b=torch.empty((B, N_HID), **b16))
            self._buf[B] = b
        return b

    def forward(self, x):
        B = x.shape[0]
        c = self._bufs(B)
        cg.gemm_bf16(x, self.Wb[0], B, N_HID, N_IN, Cb=c["H1"], bias=self.b[0], aux_out=c["Z1"],
                     epilogue=cg.EPI_BIAS_GELU)
        cg.gemm_bf16(c["H1"], self.Wb[1], B, N_HID, N_HID, Cb=c["H2"], bias=self.b[1], aux_out=c["Z2"],
                     epilogue=cg.EPI_BIAS_GELU)
        cg.gemm_bf16(c["H2"], self.Wb[2], B, N_PAD, N_HID, Cf=c["Y"], bias=self.b[2], epilogue=cg.EPI_BIAS_F32)
        return c["Y"]

    def loss_and_grad(self, target):
        B = target.shape[0]
        c = self._bufs(B)
        cg._check(cg.lib().cg_mse_loss(_p(c["Y"]), _p(target), B, N_OUT, N_PAD, _p(self.loss), _p(c["dYf"]),
                                       _p(c["dYb"]), _s()), "cg_mse_loss")
        return self.loss

    def backward(self, x):
        B = x.shape[0]
        c = self._bufs(B)
        gW1, gW2, gW3, gb1, gb2, gb3 = self.grads
        L = cg.lib()
        cg.gemm_bf16(c["dYb"], c["H2"], N_PAD, N_HID, B, transA=1, transB=1, Cf=gW3)
        cg._check(L.cg_colsum(_p(c["dYf"]), B, N_PAD, _p(gb3), _s()), "cg_colsum")
        cg.gemm_bf16(c["dYb"], self.Wb[2], B, N_HID, N_PAD, transB=1, Cf=c["dZf"], Cb=c["dZb"], aux_in=c["Z2"],
                     epilogue=cg.EPI_GELU_GRAD)
        cg.gemm_bf16(c["dZb"], c["H1"], N_HID, N_HID, B, transA=1, transB=1, Cf=gW2)
        cg._check(L.cg_colsum(_p(c["dZf"]), B, N_HID, _p(gb2), _s()), "cg_colsum")
        cg.gemm_bf16(c["dZb"], self.Wb[1], B, N_HID, N_HID, transB=1, Cf=c["dZ1f"], Cb=c["dZ1b"], aux_in=c["Z1"],
                     epilogue=cg.EPI_GELU_GRAD)
        cg.gemm_bf16(c["dZ1b"], x, N_HID, N_IN, B, transA=1, transB=1, Cf=gW1)
        cg._check(L.cg_colsum(_p(c["dZ1f"]), B, N_HID, _p(gb1), _s()), "cg_colsum")

    def adamw(self, lr=1e-3, wd=1e-4):
        self.step += 1
        for i, (p, g, m, v) in enumerate(zip(self.params, self.grads, self.m, self.v)):
            wb = self.Wb[i] if i < 3 else None
            cg._check(cg.lib().cg_adamw(_p(p), _p(g), _p(m), _p(v), p.numel(), lr, 0.9, 0.999, 1e-8,
                                        wd if i < 3 else 0.0, self.step, _p(wb), _s()), "cg_adamw")

    def predict_start(self, x, scale):
        """Starting parameters [H, 11] (FP64) for histograms with inputs x, scales scale."""
        H = x.shape[0]
        out = torch.empty((H, 3 * K_PEAKS + 2), dtype=torch.float64, device=x.device)
        chunk = 16384
        for h0 in range(0, H, chunk):
            xb = x[h0:h0 + chunk]
            Y = self.forward(xb)
            cg._check(cg.lib().cg_decode_start(_p(Y), N_PAD, _p(scale[h0:h0 + chunk]), _p(self.t_mean),
                                               _p(self.t_std), xb.shape[0], K_PEAKS, FACTOR, N_BINS, 0.0, 1.0,
                                               _p(out[h0:h0 + chunk]), _s()), "cg_decode_start")
        return out


def fit_batch(y_flat, H, theta0, n_steps=50, tol=1e-9, precision=FIT_PRECISION):
    """Batched Baker-Cousins fits of H 2048-bin histograms from theta0; returns the fitter."""
    offs = np.arange(H + 1, dtype=np.int64) * N_BINS
    b = HistBatch(y_flat, offs, np.zeros(H), np.ones(H), K_PEAKS, 1, cg.OBJ_POISSON_BC, poly_mode=0,
                  precision=precision)
    f = BatchFitter(b, FIT_MAP)
    f.init(theta0.contiguous())
    f.step(n_steps, tol)
    return f


def choose_start(y_flat, H, th_a, th_b):
    """Per histogram, the candidate start with the lower objective value
    (one batched evaluation of each candidate)."""
    offs = np.arange(H + 1, dtype=np.int64) * N_BINS
    b = HistBatch(y_flat, offs, np.zeros(H), np.ones(H), K_PEAKS, 1, cg.OBJ_POISSON_BC, poly_mode=0,
                  precision=FIT_PRECISION)
    th_a, th_b = th_a.contiguous(), th_b.contiguous()
    fa = b.objective(th_a)
    fb = b.objective(th_b)
    out = torch.empty_like(th_a)
    cg._check(cg.lib().cg_select_start(_p(fa), _p(fb), _p(th_a), _p(th_b), H, th_a.shape[1], _p(out), None, _s()),
              "cg_select_start")
    return out


def make_training_set(n_hist, chunk=65536, first_chunk=1, device="cuda", log=None, precision=FIT_PRECISION):
    """Method-generated histograms and their converged plain fits (started at
    the truth): network inputs x (bf16), scales and fitted parameters."""
    xs, ss, ts = [], [], []
    n_done, c = 0, first_chunk
    while n_done < n_hist:
        H = min(chunk, n_hist - n_done)
        d = synth.c5_batch_device(H, N_BINS, chunk=c, device=device)
        x, scale = rebin(d["y"], H)
        f = fit_batch(d["y"], H, torch.tensor(d["truth"], device=device), precision=precision)
        ok = f.states.status == cg.FIT_CONVERGED
        xs.append(x[ok])
        ss.append(scale[ok])
        ts.append(f.states.theta[ok].clone())
        if log:
            log("chunk %d: %d/%d converged" % (c, int(ok.sum()), H))
        n_done += H
        c += 1
        del d, f
    return torch.cat(xs), torch.cat(ss), torch.cat(ts)


class Trainer:
    """AdamW on the MSE of z-scored targets with a cosine-decayed learning
    rate, over shuffled minibatches of a fixed training set.

    The whole training state -- FP32 master weights and biases, Adam
    moments, the step count, the target normalisation, the epoch, the
    position inside it and the shuffling generator's state at the epoch's
    start -- goes into state_dict(); a Trainer built from it continues with
    exactly the same minibatches and kernels, so the loss curve after a
    resume is bitwise the one of an uninterrupted run."""

    def __init__(self, net, x, scale, theta, epochs=3, batch=1024, lr=1e-3, seed=0, cosine=True, log_every=50):
        self.net, self.x = net, x
        self.log_every = log_every
        self.epochs, self.batch, self.lr, self.cosine = epochs, batch, lr, cosine
        t = encode_targets(theta, scale)
        net.t_mean = t.mean(0).float().contiguous()
        w = torch.tensor(TARGET_WEIGHTS, dtype=torch.float32, device=x.device)
        # dividing the scale by w weights the squared error of target j by w_j^2
        net.t_std = (t.std(0).clamp_min(1e-6).float() / w).contiguous()
        self.tz = ((t - net.t_mean.double()) / net.t_std.double()).float().contiguous()
        self.N = x.shape[0]
        self.gen = torch.Generator(device=x.device)
        self.gen.manual_seed(seed)
        self.epoch, self.i0 = 0, 0
        self._new_epoch()
        self.curve = []

    def _new_epoch(self):
        self.gen_state = self.gen.get_state()   # the permutation of this epoch is drawn from here
        self.perm = torch.randperm(self.N, generator=self.gen, device=self.x.device)

    @property
    def total_steps(self):
        return self.epochs * (self.N // self.batch)

    def done(self):
        return self.epoch >= self.epochs

    def run(self, n_steps=None, log=None):
        """Train n_steps minibatches (None: to the end); returns the loss
        curve so far, (step, loss) at the first step and every log_every steps."""
        net = self.net
        left = n_steps
        while not self.done() and (left is None or left > 0):
            if self.i0 + self.batch > self.N:
                if log:
                    log("epoch %d: loss %.4f" % (self.epoch, self.curve[-1][1] if self.curve else float("nan")))
                self.epoch += 1
                self.i0 = 0
                if self.done():
                    break
                self._new_epoch()
                continue
            frac = net.step / max(self.total_steps, 1)
            lr_now = self.lr * (0.5 * (1.0 + math.cos(math.pi * frac)) * 0.95 + 0.05) if self.cosine else self.lr
            idx = self.perm[self.i0:self.i0 + self.batch]
            xb = self.x.index_select(0, idx).contiguous()
            tb = self.tz.index_select(0, idx).contiguous()
            net.forward(xb)
            net.loss_and_grad(tb)
            net.backward(xb)
            net.adamw(lr=lr_now)
            self.i0 += self.batch
            if net.step == 1 or net.step % self.log_every == 0:
                self.curve.append((net.step, float(net.loss)))
            if left is not None:
                left -= 1
        return self.curve

    def state_dict(self):
        net = self.net
        return {"W": [w.clone() for w in net.W], "b": [b.clone() for b in net.b],
                "m": [m.clone() for m in net.m], "v": [v.clone() for v in net.v], "step": net.step,
                "t_mean": net.t_mean.clone(), "t_std": net.t_std.clone(), "epoch": self.epoch, "i0": self.i0,
                "gen_state": self.gen_state.cpu().clone(), "curve": list(self.curve),
                "config": {"epochs": self.epochs, "batch": self.batch, "lr": self.lr, "cosine": self.cosine}}

    def load_state_dict(self, sd):
        net = self.net
        for dst, src in zip(net.W + net.b + net.m + net.v, sd["W"] + sd["b"] + sd["m"] + sd["v"]):
            dst.copy_(src)
        for w, wb in zip(net.W, net.Wb):
            cg._check(cg.lib().cg_to_bf16(_p(w), w.numel(), _p(wb), _s()), "cg_to_bf16")
        net.step = int(sd["step"])
        net.t_mean = sd["t_mean"].clone()
        net.t_std = sd["t_std"].clone()
        c = sd["config"]
        self.epochs, self.batch, self.lr, self.cosine = c["epochs"], c["batch"], c["lr"], c["cosine"]
        self.epoch, self.i0 = int(sd["epoch"]), int(sd["i0"])
        self.gen.set_state(sd["gen_state"].cpu().to(torch.uint8).clone())   # generator states are CPU byte tensors
        self._new_epoch()          # the same permutation as at the checkpoint's epoch start
        self.curve = list(sd["curve"])

    def save(self, path):
        torch.save(self.state_dict(), path)

    def load(self, path):
        self.load_state_dict(torch.load(path, map_location=self.x.device, weights_only=False))


def train(net, x, scale, theta, epochs=3, batch=1024, lr=1e-3, seed=0, log=None, cosine=True):
    """Train to the end (see Trainer); returns the loss curve."""
    return Trainer(net, x, scale, theta, epochs=epochs, batch=batch, lr=lr, seed=seed, cosine=cosine).run(log=log)


def production_fit(net, y, H, n_steps=50, tol=1e-9, precision=FIT_PRECISION, refine=True):
    """Fits of H histograms from the learned start, judged by the plain fit:
    every histogram is fitted from the network's start (sharpened on the
    full-resolution histogram when refine is set); the histograms whose fit
    did not converge within n_steps iterations are fitted again from the
    plain peak-finding heuristic start (sharpened alike), and the lower of
    the two minima is kept.  Returns dict(theta [H, P], f [H], status [H],
    iters [H], evals [H], refit (indices refitted, host), learned (the
    learned-start fitter))."""
    x, scale = rebin(y, H)
    th0 = net.predict_start(x, scale)
    if refine:
        th0 = refine_start(y, H, th0)
    fl = fit_batch(y, H, th0, n_steps, tol, precision=precision)
    st = fl.states
    theta, f = st.theta.clone(), st.f.clone()
    status, iters, evals = st.status.clone(), st.iters.clone(), st.n_eval.clone()
    idx = torch.nonzero(status != cg.FIT_CONVERGED).flatten()
    if idx.numel():
        ysub = y.view(H, N_BINS).index_select(0, idx).reshape(-1).contiguous()
        thh = heuristic_start(ysub, idx.numel())
        if refine:
            thh = refine_start(ysub, idx.numel(), thh)
        fr = fit_batch(ysub, idx.numel(), thh, n_steps, tol, precision=precision)
        rs = fr.states
        better = rs.f < f[idx]
        pick = idx[better]
        theta[pick] = rs.theta[better]
        f[pick] = rs.f[better]
        status[pick] = rs.status[better]
        iters[idx] += rs.iters
        evals[idx] += rs.n_eval
    return dict(theta=theta, f=f, status=status, iters=iters, evals=evals, refit=idx.cpu().numpy(), learned=fl)
