"""The learned window on the GPU: training kernels against the FP64 CPU
reference (gradients), training progress, checkpoints, inference, and the
learned FP32 form (window from the network, in-kernel check, fallback to the
search) against the oracle, including what the network saves.

The trained network is the committed checkpoint
paper_2502_00356_gb300/weights/window_mlp.bkw (made by train_window.py from
the oracle's labels, see oracle/make_window_labels.py)."""
import math
import os

import numpy as np
import pytest

import oracle
import paper_2502_00356_gb300 as bk
from oracle import mlp
from paper_2502_00356_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CKPT = os.path.join(ROOT, "paper_2502_00356_gb300", "weights", "window_mlp.bkw")
LOG_EPS32 = -23 * math.log(2)
F32_RTOL = 1e-5


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    bk.build()
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def small_labels():
    x, nu = inputs.kv_pairs(4096, seed=71, nu_lo=0.05, nu_hi=20.0)
    lab = oracle.window_labels(x, nu, LOG_EPS32, 1e-6)
    assert np.all(lab[:, 4] > 0)
    return x, nu, lab


def to_dev(a, dev):
    return torch.as_tensor(np.ascontiguousarray(a), device=dev)


@pytest.fixture(scope="module")
def trained(dev):
    m = bk.LearnedWindow(path=CKPT)
    return m


# Tolerances of the two training kernels: the FP32 SIMT step (relative loss
# 1e-5, gradient 2e-4 of its largest component) and the tensor-core step,
# whose hidden-layer products read TF32 operands (10 significand bits,
# relative rounding up to 2^-10 per operand): 5e-3 and 1e-2.
TRAIN_TOL = {bk.BK_TRAIN_SIMT: (1e-5, 2e-4), bk.BK_TRAIN_TENSOR: (5e-3, 1e-2)}


@pytest.mark.parametrize("path", [bk.BK_TRAIN_SIMT, bk.BK_TRAIN_TENSOR])
def test_gradient_matches_fp64_reference(dev, small_labels, path):
    x, nu, lab = small_labels
    m = bk.LearnedWindow(seed=3)
    m.set_train_path(path)
    X, V, Lb = to_dev(x, dev), to_dev(nu, dev), to_dev(lab, dev)
    m.train(X, V, Lb, steps=0)  # computes the target statistics only
    stats = m.stats()
    p = m.params().astype(np.float64)
    n = 512
    g, loss = m.grad(X[:n], V[:n], Lb[:n])
    torch.cuda.synchronize()
    U = mlp.normalise_inputs(x[:n], nu[:n])
    T = (mlp.targets_from_labels(lab[:n]) - stats[:4]) / stats[4:]
    ref_loss, ref_g = mlp.loss_and_grad(p, U, T)
    got = g.cpu().numpy().astype(np.float64)
    ltol, gtol = TRAIN_TOL[path]
    assert abs(float(loss) - ref_loss) <= ltol * ref_loss + 1e-7
    scale = np.abs(ref_g).max()
    assert np.abs(got - ref_g).max() <= gtol * scale
    # every parameter block (W1, b1, ..., b4) carries its gradient
    for a, b in ((0, 128), (128, 192), (192, 4288), (4288, 4352), (4352, 8448), (8448, 8512),
                 (8512, 8768), (8768, 8772)):
        blk = np.abs(ref_g[a:b]).max()
        assert np.abs(got[a:b] - ref_g[a:b]).max() <= 5 * gtol * blk + gtol * scale, (a, b)
    # and against central finite differences of the FP64 forward pass
    rng = np.random.default_rng(5)
    for i in rng.choice(mlp.N_PARAMS, 25, replace=False):
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (mlp.loss_only(p + e, U, T) - mlp.loss_only(p - e, U, T)) / 2e-6
        assert abs(fd - got[i]) <= gtol * scale
    assert m.params() is not None  # no tensor-core step gave up (BK_ERR_CUDA otherwise)


def test_tensor_core_and_simt_steps_agree(dev, small_labels):
    """The two training kernels on the same 1,024 samples: gradients within
    the TF32 tolerance of each other, and one Adam step apart by little."""
    x, nu, lab = small_labels
    X, V, Lb = to_dev(x, dev), to_dev(nu, dev), to_dev(lab, dev)
    grads = {}
    for path in (bk.BK_TRAIN_SIMT, bk.BK_TRAIN_TENSOR):
        m = bk.LearnedWindow(seed=6)
        m.set_train_path(path)
        m.train(X, V, Lb, steps=0)
        grads[path] = m.grad(X[:1024], V[:1024], Lb[:1024])[0].cpu().numpy().astype(np.float64)
    a, b = grads[bk.BK_TRAIN_SIMT], grads[bk.BK_TRAIN_TENSOR]
    assert np.abs(a - b).max() <= 1e-2 * np.abs(a).max()
    with pytest.raises(bk.BkError):
        bk.LearnedWindow(seed=1).set_train_path(7)


@pytest.mark.parametrize("path", [bk.BK_TRAIN_SIMT, bk.BK_TRAIN_TENSOR])
def test_training_reduces_loss(dev, small_labels, path):
    x, nu, lab = small_labels
    m = bk.LearnedWindow(seed=4)
    m.set_train_path(path)
    loss = torch.zeros(400, dtype=torch.float32, device=dev)
    m.train(to_dev(x, dev), to_dev(nu, dev), to_dev(lab, dev), steps=400, batch=1024, lr=3e-3,
            loss=loss)
    torch.cuda.synchronize()
    c = loss.cpu().numpy()
    assert np.all(np.isfinite(c))
    assert c[-50:].mean() < 0.2 * c[:10].mean()


def test_checkpoint_roundtrip_and_rejection(dev, small_labels, tmp_path):
    x, nu, lab = small_labels
    m = bk.LearnedWindow(seed=5)
    m.train(to_dev(x, dev), to_dev(nu, dev), to_dev(lab, dev), steps=20, batch=512)
    path = str(tmp_path / "w.bkw")
    m.save(path)
    m2 = bk.LearnedWindow(seed=99, path=path)
    assert np.array_equal(m.params(), m2.params())
    assert np.array_equal(m.stats(), m2.stats())
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 0xFF
    bad = str(tmp_path / "bad.bkw")
    open(bad, "wb").write(raw)
    with pytest.raises(bk.BkError):
        bk.LearnedWindow(path=bad)
    # resume: training continues from the saved step
    m2.train(to_dev(x, dev), to_dev(nu, dev), to_dev(lab, dev), steps=5, batch=512)


def test_infer_matches_fp64_forward(dev, trained):
    x, nu = inputs.kv_pairs(300, seed=72, nu_hi=20.0)
    out = trained.infer(to_dev(x, dev), to_dev(nu, dev)).cpu().numpy().astype(np.float64)
    stats = trained.stats().astype(np.float64)
    y, _ = mlp.forward(trained.params().astype(np.float64), mlp.normalise_inputs(x, nu))
    y = y * stats[4:] + stats[:4]
    want = np.stack([y[:, 0], y[:, 0] - y[:, 1], y[:, 0] + y[:, 2], np.exp(y[:, 3])], axis=1)
    assert np.abs(out - want).max() <= 1e-3 * max(1.0, np.abs(want).max())


def test_trained_network_predicts_windows(dev, trained):
    x, nu = inputs.kv_pairs(2000, seed=73, nu_hi=20.0)
    out = trained.infer(to_dev(x, dev), to_dev(nu, dev)).cpu().numpy()
    lab = oracle.window_labels(x, nu, LOG_EPS32, 1e-6)
    err_ts = np.abs(out[:, 0] - lab[:, 0])
    err_t1 = np.abs(out[:, 2] - lab[:, 2])
    assert np.median(err_ts) < 0.05 and np.median(err_t1) < 0.05


def counters(dev):
    return torch.zeros(bk.BK_NUM_COUNTERS, dtype=torch.int64, device=dev)


def test_learned_eval_accuracy_and_fallback(dev, trained):
    x, nu = inputs.kv_pairs(20_000, seed=8, nu_lo=0.05, nu_hi=20.0)
    ctr = counters(dev)
    out, lout = bk.bk_eval_ex(to_dev(x, dev), to_dev(nu, dev),
                              opts=bk.make_opts(learned=trained, counters=ctr), want_log=True)
    torch.cuda.synchronize()
    idx = np.random.default_rng(3).choice(x.size, 3000, replace=False)
    _, lref = oracle.besselk(x[idx], nu[idx], return_log=True)
    err = np.abs(np.expm1(lout.cpu().numpy()[idx] - lref))
    assert err.max() <= F32_RTOL
    c = ctr.cpu().numpy()
    assert c[bk.BK_CTR_EVALS] == 20_000 and c[bk.BK_CTR_FAIL] == 0
    assert c[bk.BK_CTR_FALLBACK] <= 0.1 * 20_000


def test_learned_gain_over_search(dev, trained):
    """What the network saves: the learned window replaces the per-point root
    finding (the Newton iterations drop to those of the fallback points)
    while the node count stays within a few per cent of the searched window."""
    x, nu = inputs.kv_pairs(50_000, seed=9, nu_lo=0.05, nu_hi=20.0)
    X, V = to_dev(x, dev), to_dev(nu, dev)
    c_s, c_l = counters(dev), counters(dev)
    bk.bk_eval_ex(X, V, opts=bk.make_opts(compute=bk.BK_F32, counters=c_s))
    bk.bk_eval_ex(X, V, opts=bk.make_opts(learned=trained, counters=c_l))
    torch.cuda.synchronize()
    s, l = c_s.cpu().numpy(), c_l.cpu().numpy()
    it_s = s[bk.BK_CTR_ITERS] + s[bk.BK_CTR_PEAK_ITERS]
    it_l = l[bk.BK_CTR_ITERS] + l[bk.BK_CTR_PEAK_ITERS]
    assert it_l <= 0.15 * it_s
    assert l[bk.BK_CTR_NODES] <= 1.15 * s[bk.BK_CTR_NODES]


def test_corrupted_network_falls_back_and_stays_correct(dev, trained):
    m = bk.LearnedWindow(seed=0, path=CKPT)
    m.params(np.zeros(bk.N_MLP_PARAMS, dtype=np.float32))  # predicts the mean window everywhere
    x, nu = inputs.kv_pairs(3000, seed=10, nu_hi=20.0)
    ctr = counters(dev)
    _, lout = bk.bk_eval_ex(to_dev(x, dev), to_dev(nu, dev),
                            opts=bk.make_opts(learned=m, counters=ctr), want_log=True)
    torch.cuda.synchronize()
    _, lref = oracle.besselk(x, nu, return_log=True)
    assert np.abs(np.expm1(lout.cpu().numpy() - lref)).max() <= F32_RTOL
    assert ctr.cpu().numpy()[bk.BK_CTR_FALLBACK] > 0.5 * 3000


def test_learned_matern_and_batched(dev, trained):
    n, beta, nu = 3000, 0.1, 1.7
    locs = inputs.morton_sorted(inputs.jittered_grid(n, seed=11))
    L = to_dev(locs, dev)
    ctr = counters(dev)
    out = torch.empty((n, n), dtype=torch.float32, device=dev)
    bk.bk_matern_tile(L, 1.0, beta, nu, out=out, opts=bk.make_opts(learned=trained, counters=ctr))
    torch.cuda.synchronize()
    I, J = inputs.entry_sample(n, 3000, seed=12)
    got = out[torch.as_tensor(J, device=dev), torch.as_tensor(I, device=dev)].double().cpu().numpy()
    want = oracle.matern_entries(locs, I, J, 1.0, beta, nu)
    big = want >= 1e-30
    assert np.abs(got[big] / want[big] - 1).max() <= F32_RTOL
    assert ctr.cpu().numpy()[bk.BK_CTR_FALLBACK] <= 0.1 * n * n / 2
    # batched persistent form with the learned window equals the single call
    o2 = torch.empty_like(out)
    d = bk.make_descs([(L, 1.0, beta, nu, o2)])
    plan = bk.BatchedPlan([n], dtype=torch.float32, opts=bk.make_opts(learned=trained))
    bk.bk_matern_batched(d, plan)
    torch.cuda.synchronize()
    rel = ((o2.double() - out.double()).abs() / out.double().abs().clamp_min(1e-30)).max()
    # the same entries from another kernel: their windows may differ in the
    # last bits (FMA contraction), and with them N; two FP32-form results
    # agree to twice the form's typical error (~1e-6), far inside 1e-5
    assert float(rel) <= 2e-6


def test_learned_needs_weights_and_fp32(dev):
    m = bk.LearnedWindow(seed=1)  # never trained: no statistics
    x = torch.ones(4, dtype=torch.float64, device=dev)
    with pytest.raises(bk.BkError) as e:
        bk.bk_eval_ex(x, x, opts=bk.make_opts(learned=m))
    assert e.value.status == bk.BK_ERR_NOT_LOADED
