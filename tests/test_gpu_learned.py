"""Learned gridding kernel on the GPU: the training gradient against FP64 finite
differences of the oracle's image, and the gain over the Gaussian after training."""
import math

import numpy as np
import pytest

import oracle
from oracle import OracleConfig
from paper_2301_06061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_06061_gb300 import autograd, build, learned, wst

    build.build()
    wst.load_library()
    return wst, learned, autograd


def test_training_gradient_matches_oracle_finite_differences(mods):
    """d loss / d table through wst_image + wst_kernel_grad + the torch grid correction,
    against central differences of the same loss evaluated with the FP64 oracle."""
    wst, learned, autograd = mods
    n, fov, n_w, W, per = 64, 0.1, 2, 8, 8
    L = W * per + 1
    work = synth.learned_sky(7, n=n, fov=fov, n_vis=400)
    vis = oracle.predict_points(work.u, work.v, work.w, work.sky.l, work.sky.m, work.sky.flux).astype(np.complex64)
    rng = np.random.default_rng(1)
    pa = rng.integers(n // 4, 3 * n // 4, 40).astype(np.int32)
    pb = rng.integers(n // 4, 3 * n // 4, 40).astype(np.int32)
    target = oracle.dft_pixels(work.u, work.v, work.w, vis, n, fov, pa, pb)
    tab0 = np.exp(-np.linspace(-4, 4, L) ** 2 / (2 * 0.925**2))

    def loss_oracle(t):
        cfg = OracleConfig(n, fov, n_w, -200.0, 200.0, W, "table", 0.0, t)
        d = oracle.image_pixels(cfg, work.u, work.v, work.w, vis, pa, pb)
        return np.sum(np.abs(d - target) ** 2) / np.sum(np.abs(target) ** 2)

    cfg = wst.Config(n=n, fov=fov, n_w=n_w, w_min=-200.0, w_max=200.0, support=W,
                     kernel=wst.WST_KERNEL_TABLE, ktable_len=L)
    plan = wst.Plan(cfg)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    M = torch.from_numpy(learned.correction_matrix(n, W, L)).cuda()
    table = torch.tensor(tab0, dtype=torch.float32, device="cuda", requires_grad=True)
    U = autograd.kernel_image(table, plan, dev(work.u), dev(work.v), dev(work.w), dev(vis))[0]
    ghat = (M @ table.double()).float()
    ia, ib = dev(pa).long(), dev(pb).long()
    D = U[ib, ia] / (ghat[ia] * ghat[ib])
    tgt = dev(target.astype(np.complex64))
    loss = torch.sum(torch.abs(D - tgt) ** 2) / torch.sum(torch.abs(tgt) ** 2)
    loss.backward()
    g = table.grad.cpu().numpy()
    h = 1e-4
    scale = np.abs(g).max()
    for i in (0, 9, L // 2 - 3, L // 2, L - 12, L - 1):
        tp, tm = tab0.copy(), tab0.copy()
        tp[i] += h
        tm[i] -= h
        fd = (loss_oracle(tp) - loss_oracle(tm)) / (2 * h)
        assert abs(fd - g[i]) < 2e-3 * scale, (i, fd, g[i])


def test_learned_kernel_beats_gaussian_at_equal_support(mods):
    """A short training (300 synthetic skies) already lowers the image error against the
    direct transform on held-out skies below the W = 8 Gaussian's."""
    wst, learned, _ = mods
    torch.manual_seed(11)
    mlp = learned.KernelMLP(8).cuda()
    gauss = learned.gaussian_table(8, wst.DEFAULT_SIGMA[8], device="cuda")
    learned.fit_to_table(mlp, gauss, 8, 1024, steps=1000)
    tr = learned.Trainer(n_vis=50_000, pixels=1024)
    tr.train(mlp, range(300))
    held_out = range(2_000_000, 2_000_020)
    err_gauss = tr.evaluate(gauss, held_out)
    err_learned = tr.evaluate(learned.tabulate(mlp, 8, 1024, "cuda").detach(), held_out)
    assert math.isfinite(err_learned)
    assert err_learned < 0.7 * err_gauss, (err_learned, err_gauss)
