"""BF16 tensor-core kernels of the learned-start network against CPU FP32
references computed from the same BF16-rounded inputs."""
import numpy as np
import pytest
import torch

from paper_2203_06139_gb300 import cg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _bf(shape, seed, dev, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(shape, generator=g) * scale).to(torch.bfloat16).to(dev)


@pytest.mark.parametrize("M,N,K,tA,tB", [(200, 512, 256, 0, 0), (300, 16, 512, 0, 0), (128, 128, 64, 0, 0),
                                         (257, 72, 200, 0, 0), (1000, 24, 520, 0, 0), (4096, 512, 512, 0, 0),
                                         (64, 300, 130, 0, 0), (257, 512, 320, 0, 1), (512, 256, 200, 1, 1),
                                         (96, 40, 130, 1, 0)])
def test_gemm_matches_fp32_reference(dev, M, N, K, tA, tB):
    """K-major operands with rows of a multiple of 8 elements take the TMA
    kernels (persistent for N >= 128; tails in M, N and K included);
    transposed operands and K = 130 take the register-staged kernel."""
    A = _bf((K, M) if tA else (M, K), 1, dev)
    B = _bf((K, N) if tB else (N, K), 2, dev)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    cg.gemm_bf16(A, B, M, N, K, transA=tA, transB=tB, Cf=C, err=err)
    torch.cuda.synchronize()
    a = A.float().cpu()
    b = B.float().cpu()
    ref = (a.T if tA else a) @ (b if tB else b.T)
    assert int(err.item()) == 0
    torch.testing.assert_close(C.cpu(), ref, rtol=1e-4, atol=1e-4 * float(ref.abs().max()))


@pytest.mark.parametrize("M,N,K", [(8192, 1024, 256), (20000, 512, 192), (40000, 200, 136), (300, 2048, 64)])
def test_gemm_persistent_many_tiles_per_cta(dev, M, N, K):
    """The persistent kernel (N >= 128) with more output tiles than SMs:
    both TMEM accumulators of a CTA alternate, and the stage ring runs across
    tiles; tails in M, N and K."""
    A = _bf((M, K), 5, dev)
    B = _bf((N, K), 6, dev)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    cg.gemm_bf16(A, B, M, N, K, Cf=C, err=err)
    torch.cuda.synchronize()
    ref = A.float().cpu() @ B.float().cpu().T
    assert int(err.item()) == 0
    torch.testing.assert_close(C.cpu(), ref, rtol=1e-4, atol=1e-4 * float(ref.abs().max()))


@pytest.mark.slow
@pytest.mark.parametrize("M,N,K", [(65536, 512, 512), (8192, 8192, 8192)])
def test_gemm_full_size_sampled_rows(dev, M, N, K):
    """The benchmarked shapes: sampled rows of C (first, last and spread
    between) against an FP32 reference of the same BF16 operands."""
    g = torch.Generator(device=dev).manual_seed(9)
    A = torch.randn((M, K), generator=g, device=dev).to(torch.bfloat16)
    B = torch.randn((N, K), generator=g, device=dev).to(torch.bfloat16)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    cg.gemm_bf16(A, B, M, N, K, Cf=C, err=err)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    rows = torch.tensor(sorted({0, M - 1, 127, 128, M // 2, M // 3} | set(range(1000, M, M // 24))), device=dev)
    ref = A[rows].float().cpu() @ B.float().cpu().T
    torch.testing.assert_close(C[rows].cpu(), ref, rtol=1e-4, atol=1e-4 * float(ref.abs().max()))
    assert not torch.isnan(C).any()


def test_gemm_persistent_epilogues(dev):
    M, N, K = 3000, 384, 256
    A, B = _bf((M, K), 7, dev), _bf((N, K), 8, dev)
    bias = torch.randn(N, device=dev)
    z = torch.empty((M, N), device=dev)
    h = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
    cg.gemm_bf16(A, B, M, N, K, Cb=h, bias=bias, aux_out=z, epilogue=cg.EPI_BIAS_GELU)
    ref_z = A.float() @ B.float().T + bias
    torch.testing.assert_close(z, ref_z, rtol=1e-4, atol=1e-3)
    torch.testing.assert_close(h.float(), torch.nn.functional.gelu(ref_z).bfloat16().float(), rtol=1e-2, atol=1e-2)
    dz = torch.empty((M, N), device=dev)
    cg.gemm_bf16(A, B, M, N, K, Cf=dz, aux_in=z, epilogue=cg.EPI_GELU_GRAD)
    zz = z.clone().requires_grad_(True)
    torch.nn.functional.gelu(zz).backward(A.float() @ B.float().T)
    torch.testing.assert_close(dz, zz.grad, rtol=1e-3, atol=1e-3)


def test_gemm_epilogues(dev):
    M, N, K = 150, 96, 128
    A, B = _bf((M, K), 3, dev), _bf((N, K), 4, dev)
    bias = torch.randn(N, device=dev)
    z = torch.empty((M, N), device=dev)
    h = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
    cg.gemm_bf16(A, B, M, N, K, Cb=h, bias=bias, aux_out=z, epilogue=cg.EPI_BIAS_GELU)
    ref_z = A.float() @ B.float().T + bias
    torch.testing.assert_close(z, ref_z, rtol=1e-4, atol=1e-3)
    torch.testing.assert_close(h.float(), torch.nn.functional.gelu(ref_z).bfloat16().float(), rtol=1e-2, atol=1e-2)
    dz = torch.empty((M, N), device=dev)
    cg.gemm_bf16(A, B, M, N, K, Cf=dz, aux_in=z, epilogue=cg.EPI_GELU_GRAD)
    zz = z.clone().requires_grad_(True)
    torch.nn.functional.gelu(zz).backward(A.float() @ B.float().T)
    torch.testing.assert_close(dz, zz.grad, rtol=1e-3, atol=1e-3)


# --------------------------------------------------------------------------
# learned start: rebinning, heuristic start, network gradients, training
# --------------------------------------------------------------------------
from paper_2203_06139_gb300 import learned_start as ls  # noqa: E402
from paper_2203_06139_gb300 import synth  # noqa: E402
import numpy as np  # noqa: E402


def test_rebin_normalize(dev):
    d = synth.c5_batch(H=37, n_bins=2048)
    y = torch.tensor(d["y"], device=dev)
    x, scale = ls.rebin(y, 37)
    r = d["y"].reshape(37, 256, 8).sum(2)
    m = r.max(1)
    np.testing.assert_allclose(scale.cpu().numpy(), m, rtol=1e-6)
    np.testing.assert_allclose(x.float().cpu().numpy(), r / m[:, None], rtol=1e-2, atol=1e-3)


def test_heuristic_start_finds_the_peaks(dev):
    """Where the three peaks are well separated (gaps above 2.5 (s_i + s_j)),
    the heuristic locates each to within 4 rebinned bins; overlapping peaks
    are beyond a local-maximum search."""
    H = 256
    d = synth.c5_batch(H=H, n_bins=2048)
    y = torch.tensor(d["y"], device=dev)
    th = ls.heuristic_start(y, H).cpu().numpy()
    mu_t, s_t = d["truth"][:, 1:9:3], d["truth"][:, 2:9:3]
    sep = np.ones(H, dtype=bool)
    for k in range(3):
        for q in range(3):
            if q != k:
                sep &= np.abs(mu_t[:, k] - mu_t[:, q]) > 2.5 * (s_t[:, k] + s_t[:, q])
    assert sep.sum() > 40
    err = np.abs(th[:, 1:9:3] - mu_t)
    assert np.mean(err[sep] < 4 * 8 / 2048) > 0.95
    assert np.all(th[:, 0:9:3] > 0) and np.all(th[:, 2:9:3] > 0)


def _heuristic_reference(y, factor, lo, hi, K):
    """The heuristic start of cg_heuristic_start for one histogram, in the
    order of operations its definition fixes (sums in bin order, products and
    sums rounded separately)."""
    nr = len(y) // factor
    r = np.zeros(nr)
    for i in range(factor):
        r = r + y[i::factor][:nr]
    t = np.zeros(nr)
    c = np.zeros(nr)
    for d in range(-2, 3):
        q = np.arange(nr) + d
        ok = (q >= 0) & (q < nr)
        t = np.where(ok, t + r[np.clip(q, 0, nr - 1)], t)
        c = c + ok
    s = t / c
    seg = max(nr // 8, 1)
    jl = int(np.argmin(s[:seg]))
    jr = nr - seg + int(np.argmin(s[nr - seg:]))
    xl, xr = jl + 0.5, jr + 0.5
    slope = (s[jr] - s[jl]) / (xr - xl) if jr != jl else 0.0
    b_at0 = s[jl] - slope * xl
    res = s - (b_at0 + slope * (np.arange(nr) + 0.5))
    wr = (hi - lo) / nr
    pk = []
    for _ in range(min(K, 8)):
        best = -1
        for j in range(1, nr - 1):
            if not (res[j] >= res[j - 1] and res[j] >= res[j + 1]):
                continue
            if any(abs(j - q[0]) < 3 for q in pk):
                continue
            if best < 0 or res[j] > res[best]:
                best = j
        if best < 0 or not res[best] > 0.0:
            break
        half = 0.5 * res[best]
        a = b = best
        while a > 0 and res[a] > half:
            a -= 1
        while b < nr - 1 and res[b] > half:
            b += 1
        fw = max(float(b - a), 1.0)
        pk.append((best, res[best] / factor, fw * wr / 2.3548200450309493))
    mu = [lo + (j + 0.5) * wr for j, _, _ in pk]
    A = [a for _, a, _ in pk]
    sg = [w for _, _, w in pk]
    for k in range(len(pk), K):
        mu.append(lo + (hi - lo) * (k + 0.5) / K)
        A.append(1.0)
        sg.append(2.0 * wr)
    order = sorted(range(K), key=lambda k: (mu[k], k))
    th = []
    for k in order:
        th += [A[k], mu[k], sg[k]]
    per_bin = 1.0 / factor
    th += [(b_at0 - slope * lo / wr) * per_bin, slope / wr * per_bin]
    return np.array(th)


def test_heuristic_start_matches_its_definition(dev):
    """Bit for bit against the reference written from the header's definition,
    on c5-like histograms plus a flat, an empty and a one-peak histogram (the
    missing peaks are filled in)."""
    H = 300
    d = synth.c5_batch(H=H, n_bins=2048, index=9)
    y = d["y"].reshape(H, 2048).copy()
    y[0] = 50.0
    y[1] = 0.0
    xc = (np.arange(2048) + 0.5) / 2048
    y[2] = np.round(20.0 + 3000.0 * np.exp(-0.5 * ((xc - 0.3) / 0.02) ** 2))
    th = ls.heuristic_start(torch.tensor(y.reshape(-1), device=dev), H).cpu().numpy()
    for h in range(H):
        ref = _heuristic_reference(y[h], 8, 0.0, 1.0, 3)
        assert np.array_equal(th[h], ref), (h, th[h], ref)


def _ref_mlp(net, x, target):
    """Plain PyTorch FP32 forward/backward with BF16 rounding at the kernels' points."""
    bf = lambda t: t.bfloat16().float()
    W = [w.bfloat16().float() for w in net.W]
    b = net.b
    xf = x.float()
    Z1 = xf @ W[0].T + b[0]
    H1 = bf(torch.nn.functional.gelu(Z1))
    Z2 = H1 @ W[1].T + b[1]
    H2 = bf(torch.nn.functional.gelu(Z2))
    Y = H2 @ W[2].T + b[2]
    B = x.shape[0]
    d = torch.zeros_like(Y)
    d[:, :11] = Y[:, :11] - target
    loss = (d[:, :11] ** 2).mean()
    dY = 2 * d / (B * 11)
    gW3 = bf(dY).T @ H2
    dH2 = bf(dY) @ W[2]
    Z2r = Z2.clone().requires_grad_(True)
    torch.nn.functional.gelu(Z2r).backward(dH2)
    dZ2 = Z2r.grad
    gW2 = bf(dZ2).T @ H1
    dH1 = bf(dZ2) @ W[1]
    Z1r = Z1.clone().requires_grad_(True)
    torch.nn.functional.gelu(Z1r).backward(dH1)
    dZ1 = Z1r.grad
    gW1 = bf(dZ1).T @ xf
    return Y, loss, [gW1, gW2, gW3, dZ1.sum(0), dZ2.sum(0), dY.sum(0)]


def test_mlp_forward_backward_vs_reference(dev):
    net = ls.MLP(seed=3)
    g = torch.Generator().manual_seed(4)
    x = torch.rand((200, 256), generator=g).bfloat16().to(dev)
    t = torch.randn((200, 11), generator=g).to(dev)
    Y = net.forward(x)
    loss = net.loss_and_grad(t)
    net.backward(x)
    torch.cuda.synchronize()
    Yr, lr_, gr = _ref_mlp(net, x, t)
    # the bars of the network's parity: outputs within 1e-3 and weight
    # gradients within 1e-2 (normwise: largest deviation over the largest
    # entry) of an FP32 reference with BF16 rounding at the kernel's points;
    # what remains is FP32 summation order and the rare BF16 rounding that
    # tips the other way
    assert float((Y - Yr).abs().max()) <= 1e-3 * float(Yr.abs().max())
    assert abs(float(loss) - float(lr_)) <= 1e-4 * float(lr_)
    for got, ref in zip(net.grads, gr):
        scale = float(ref.abs().max())
        assert float((got - ref).abs().max()) <= 1e-2 * scale, (got.shape, float((got - ref).abs().max()), scale)


def test_training_reduces_loss(dev):
    d = synth.c5_batch_device(16384, chunk=91, device=dev)
    x, scale = ls.rebin(d["y"], 16384)
    theta = torch.tensor(d["truth"], device=dev)
    net = ls.MLP(seed=0)
    curve = ls.train(net, x, scale, theta, epochs=10, batch=256, lr=1e-3)
    assert curve[0][0] == 1 and net.step == 640
    assert curve[-1][1] < 0.6 * curve[0][1], curve[:3] + curve[-3:]


def _ref_refine(y, lo, hi, K, th, sweeps, half):
    """The start refinement restated plainly (see cg.h, cg_refine_start)."""
    import math
    n = len(y)
    h = (hi - lo) / n
    A = [th[3 * k] for k in range(K)]
    mu = [th[3 * k + 1] for k in range(K)]
    s = [abs(th[3 * k + 2]) for k in range(K)]
    b0, b1 = th[3 * K], th[3 * K + 1]

    def sort():
        order = sorted(range(K), key=lambda k: mu[k])
        return [A[k] for k in order], [mu[k] for k in order], [s[k] for k in order]
    A, mu, s = sort()
    for _ in range(sweeps):
        for k in range(K):
            w = half * max(s[k], 4.0 * h)
            if not (math.isfinite(mu[k]) and math.isfinite(w) and w > 0.0):
                continue
            a0 = math.floor(((mu[k] - w) - lo) / h)
            a1 = math.ceil(((mu[k] + w) - lo) / h)
            i0 = 0 if a0 < 0 else (n if a0 > n - 1 else int(a0))
            i1 = n - 1 if a1 > n - 1 else (-1 if a1 < 0 else int(a1))
            S0 = S1 = S2 = 0.0
            for i in range(i0, i1 + 1):
                x = lo + (i + 0.5) * h
                dx = x - mu[k]
                if not abs(dx) <= w:
                    continue
                r = y[i] - (b0 + b1 * x)
                for j in range(K):
                    if j != k:
                        z = (x - mu[j]) / s[j]
                        r = r - A[j] * math.exp(-0.5 * (z * z))
                if not r > 0.0:
                    continue
                S0 += r
                S1 += r * dx
                S2 += (r * dx) * dx
            if not S0 > 0.0:
                continue
            m1 = S1 / S0
            var = max(S2 / S0 - m1 * m1, (0.5 * h) * (0.5 * h))
            z = min(max(w / math.sqrt(var), 0.5), 10.0)
            phi = 0.3989422804014327 * math.exp(-0.5 * (z * z))
            frac = 1.0 - (2.0 * z * phi) / math.erf(z * 0.7071067811865476)
            s2 = math.sqrt(var / frac)
            cover = math.erf((w / s2) * 0.7071067811865476)
            A[k] = (S0 * h) / ((s2 * 2.5066282746310002) * cover)
            mu[k] = mu[k] + m1
            s[k] = s2
        A, mu, s = sort()
    out = []
    for k in range(K):
        out += [A[k], mu[k], s[k]]
    return np.array(out + [b0, b1])


def test_refine_start_matches_its_definition(dev):
    """cg_refine_start on the heuristic starts of 12 histograms against the
    plain restatement above (sums in another order, exp and erf from
    another library: agreement to 1e-9)."""
    d = synth.c5_batch_device(12, chunk=93, device=dev)
    th = ls.heuristic_start(d["y"], 12)
    out = ls.refine_start(d["y"], 12, th)
    torch.cuda.synchronize()
    y = d["y"].view(12, ls.N_BINS).cpu().numpy()
    th, out = th.cpu().numpy(), out.cpu().numpy()
    for h in range(12):
        ref = _ref_refine(y[h], 0.0, 1.0, 3, th[h], ls.REFINE_SWEEPS, ls.REFINE_HALF_WIDTH)
        np.testing.assert_allclose(out[h], ref, rtol=1e-9, atol=1e-12)
    # the start moves: peaks centred and sized on the full-resolution counts
    assert np.any(np.abs(out[:, 1:9:3] - th[:, 1:9:3]) > 1e-6)


def test_training_checkpoint_resume_is_bitwise(dev, tmp_path):
    """A training run checkpointed part-way (weights, Adam moments, step,
    target normalisation, epoch position, shuffling generator) and resumed
    by a fresh Trainer on a differently initialised network follows the
    uninterrupted run's loss curve and ends at its weights, bit for bit."""
    d = synth.c5_batch_device(8192, chunk=92, device=dev)
    x, scale = ls.rebin(d["y"], 8192)
    theta = torch.tensor(d["truth"], device=dev)
    net = ls.MLP(seed=1)
    tr = ls.Trainer(net, x, scale, theta, epochs=3, batch=256, lr=1e-3, log_every=1)
    tr.run(40)                                  # 32 steps per epoch: the checkpoint falls inside epoch 1
    ck = tmp_path / "train.pt"
    tr.save(ck)
    tr.run()
    curve = list(tr.curve)
    W_end = [w.clone() for w in net.W] + [b.clone() for b in net.b]
    assert net.step == 96 and len(curve) == 96
    net2 = ls.MLP(seed=7)
    tr2 = ls.Trainer(net2, x, scale, theta, epochs=1, batch=128, lr=5e-3, seed=123, log_every=1)
    tr2.load(ck)
    tr2.run()
    assert net2.step == 96
    assert tr2.curve == curve                   # float losses compared exactly
    for a, b in zip(W_end, net2.W + net2.b):
        assert torch.equal(a, b)


@pytest.mark.slow
def test_learned_start_gains_over_the_heuristic(dev):
    """What the trained network adds to the method (trained here on 262,144
    method-generated fits, judged on 4096 held-out histograms): the
    production path (network start refined on the full-resolution
    histogram, refit from the refined heuristic start where that fit did not
    converge, lower minimum kept) reaches the minimum of the fit started at
    the generating truth in more histograms than the refined heuristic start
    alone, converges at least as many, and ends lower more often than
    higher."""
    x, scale, theta = ls.make_training_set(262144)
    net = ls.MLP(seed=0)
    ls.train(net, x, scale, theta, epochs=6, lr=2e-3)
    H = 4096
    d = synth.c5_batch_device(H, ls.N_BINS, chunk=0, device=dev)
    y = d["y"]
    Ft = ls.fit_batch(y, H, torch.tensor(d["truth"], device=dev), 50, 1e-9).states.f.cpu().numpy()
    fh = ls.fit_batch(y, H, ls.refine_start(y, H, ls.heuristic_start(y, H)), 50, 1e-9)
    pr = ls.production_fit(net, y, H, 50, 1e-9)
    Fh, Fp = fh.states.f.cpu().numpy(), pr["f"].cpu().numpy()
    at_truth = lambda F: float(np.mean(np.abs(F - Ft) <= 1e-6 * np.abs(Ft)))
    assert at_truth(Fp) > at_truth(Fh) + 0.03, (at_truth(Fp), at_truth(Fh))
    assert int((pr["status"] == cg.FIT_CONVERGED).sum()) >= int((fh.states.status == cg.FIT_CONVERGED).sum())
    lower, higher = int((Fp < Fh * (1 - 1e-6)).sum()), int((Fp > Fh * (1 + 1e-6)).sum())
    assert lower > 2 * higher, (lower, higher)
