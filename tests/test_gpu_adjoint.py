"""GPU parity of the adjoint (degridding), the autograd binding, the tabulated-kernel
gradient and the direct transform (the accuracy reference), against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from oracle import OracleConfig
from paper_2301_06061_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def wst():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_06061_gb300 import build, wst as w

    build.build()
    w.load_library()
    return w


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel_err(gpu, ref):
    ref = np.asarray(ref)
    return float(np.abs(np.asarray(gpu, dtype=np.complex128) - ref).max() / np.abs(ref).max())


def case(n=128, n_vis=2000, seed=0, fov=0.1):
    rng = np.random.default_rng(seed)
    u, v, w = synth.disk_uvw(n_vis, 0.45 * n / fov, 200.0, rng)
    vis = synth.random_visibilities(n_vis, rng)
    wt = rng.uniform(0.5, 2.0, n_vis).astype(np.float32)
    return u, v, w, vis, wt, rng


@pytest.mark.parametrize("n,n_w,chunk,correct", [(128, 4, 0, True), (128, 4, 3, False), (256, 3, 1, True),
                                                 (64, 1, 0, True), (2048, 2, 0, True), (16384, 2, 1, False)])
def test_degrid_matches_oracle(wst, n, n_w, chunk, correct):
    u, v, w, vis, wt, rng = case(n=n, seed=n + n_w)
    cfg = wst.Config(n=n, fov=0.1, n_w=n_w, w_min=-200.0, w_max=200.0, planes_per_chunk=chunk)
    plan = wst.Plan(cfg)
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis), dev(wt))
    y = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    flags = 0 if correct else wst.WST_NO_CORRECTION
    got = plan.degrid(dev(y[None]), flags=flags).cpu().numpy()
    ocfg = OracleConfig(n, 0.1, n_w, -200.0, 200.0, 7)
    ref = oracle.degrid(ocfg, u, v, w, vis, y, wt, correct=correct)
    assert rel_err(got, ref) < TOL


def test_degrid_dropped_get_zero(wst):
    n = 64
    u = np.array([0.0, 9000.0, 10.0], np.float32)
    v = np.zeros(3, np.float32)
    w = np.zeros(3, np.float32)
    vis = np.ones(3, np.complex64)
    vis[2] = np.nan
    plan = wst.Plan(wst.Config(n=n, fov=0.1, n_w=1, w_min=-1.0, w_max=1.0))
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis))
    got = plan.degrid(torch.ones((1, n, n), dtype=torch.complex64, device="cuda")).cpu().numpy()
    assert got[0] != 0 and got[1] == 0 and got[2] == 0


def test_dot_product_identity_on_gpu(wst):
    """<y, A x> = <A^H y, x> with both sides computed by the GPU.  Without the grid
    correction FP32 rounding is uniform (1e-5); with it, the corner factors C_a C_b
    (up to ~2e3 for W = 7) weight the rounding of the corner pixels (1e-4)."""
    n = 256
    u, v, w, vis, wt, rng = case(n=n, n_vis=5000, seed=4)
    plan = wst.Plan(wst.Config(n=n, fov=0.1, n_w=5, w_min=-200.0, w_max=200.0, planes_per_chunk=2))
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis), dev(wt))
    y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    for flags, tol in ((wst.WST_NO_CORRECTION, 1e-5), (0, 1e-4)):
        ax = plan.image(flags=flags)[0].cpu().numpy().astype(np.complex128)
        ahy = plan.degrid(dev(y.astype(np.complex64)[None]), flags=flags).cpu().numpy().astype(np.complex128)
        lhs = np.vdot(y, ax)
        rhs = np.vdot(ahy, vis.astype(np.complex128))
        assert abs(lhs - rhs) < tol * abs(lhs), (flags, abs(lhs - rhs) / abs(lhs))


def test_autograd_backward_is_oracle_adjoint(wst):
    from paper_2301_06061_gb300 import autograd

    n = 128
    u, v, w, vis, wt, rng = case(n=n, seed=6)
    plan = wst.Plan(wst.Config(n=n, fov=0.1, n_w=4, w_min=-200.0, w_max=200.0))
    y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    V = dev(vis).requires_grad_(True)
    D = autograd.image(V, plan, dev(u), dev(v), dev(w), dev(wt))
    loss = torch.real(torch.sum(torch.conj(dev(y.astype(np.complex64))) * D[0]))
    loss.backward()
    # d Re<y, A V> / d V* convention of torch: grad = A^H y
    ref = oracle.degrid(OracleConfig(n, 0.1, 4, -200.0, 200.0, 7), u, v, w, vis, y, wt)
    assert rel_err(V.grad.cpu().numpy(), ref) < TOL


def test_autograd_gradcheck_finite_differences(wst):
    """torch.autograd.gradcheck against central differences, eps = 1e-3."""
    from paper_2301_06061_gb300 import autograd

    n = 64
    u, v, w, vis, wt, rng = case(n=n, n_vis=24, seed=8)
    plan = wst.Plan(wst.Config(n=n, fov=0.1, n_w=2, w_min=-200.0, w_max=200.0))
    du, dv, dw = dev(u), dev(v), dev(w)
    x = dev(vis.astype(np.complex128)).requires_grad_(True)
    fn = lambda t: autograd.image(t, plan, du, dv, dw)
    # the forward runs in FP32: central differences carry ~1e-7 |D| / eps of rounding
    assert torch.autograd.gradcheck(fn, (x,), eps=1e-3, atol=2e-2, rtol=1e-3, fast_mode=True,
                                    nondet_tol=1e-4)


@pytest.mark.parametrize("n", [128, 2048])
def test_kernel_grad_matches_oracle(wst, n):
    W = 8
    L = W * 32 + 1
    u, v, w, vis, wt, rng = case(n=n, n_vis=1500, seed=10)
    xs = np.linspace(-W / 2, W / 2, L)
    tab = (np.exp(-xs**2 / (2 * 0.925**2)) * (1 + 0.05 * np.sin(xs))).astype(np.float32)
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-200.0, w_max=200.0, support=W, kernel=wst.WST_KERNEL_TABLE,
                     ktable_len=L, planes_per_chunk=2)
    plan = wst.Plan(cfg)
    plan.set_kernel_table(dev(tab))
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis), dev(wt))
    dU = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    got = plan.kernel_grad(dev(dU[None])).cpu().numpy()
    ocfg = OracleConfig(n, 0.1, 3, -200.0, 200.0, W, "table", 0.0, tab.astype(np.float64))
    ref = oracle.kernel_grad(ocfg, u, v, w, vis, dU, wt)
    assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()


def test_dft_matches_oracle(wst):
    n, fov = 512, 0.3
    rng = np.random.default_rng(12)
    u, v, w = synth.disk_uvw(20000, 0.45 * n / fov, 3000.0, rng)
    vis = synth.random_visibilities(20000, rng)
    wt = rng.uniform(0.5, 2.0, 20000).astype(np.float32)
    pa = rng.integers(0, n, 300).astype(np.int32)
    pb = rng.integers(0, n, 300).astype(np.int32)
    out = torch.empty(300, dtype=torch.complex64, device="cuda")
    wst.wst_dft(dev(u), dev(v), dev(w), dev(vis), n, fov, dev(pa), dev(pb), out, weight=dev(wt))
    ref = oracle.dft_pixels(u, v, w, vis, n, fov, pa, pb, wt)
    assert rel_err(out.cpu().numpy(), ref) < TOL


def test_predict_matches_oracle(wst):
    rng = np.random.default_rng(13)
    u, v, w = synth.disk_uvw(5000, 9000.0, 2000.0, rng)
    sky = synth.power_law_sky(37, 0.2, 0.01, 1.0, rng)
    out = torch.empty(5000, dtype=torch.complex64, device="cuda")
    wst.wst_predict_points(dev(u), dev(v), dev(w), dev(sky.l), dev(sky.m), dev(sky.flux), out)
    ref = oracle.predict_points(u, v, w, sky.l, sky.m, sky.flux)
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-5 * np.abs(sky.flux).sum()


def test_autograd_two_forwards_on_one_plan_before_backward(wst):
    """Each backward differentiates its own forward, also when a second forward has
    rebound the plan in between (the binding is restored from the saved inputs)."""
    from paper_2301_06061_gb300 import autograd

    n = 128
    plan = wst.Plan(wst.Config(n=n, fov=0.1, n_w=4, w_min=-200.0, w_max=200.0))
    ocfg = OracleConfig(n, 0.1, 4, -200.0, 200.0, 7)
    cases, outs = [], []
    for seed in (21, 22):
        u, v, w, vis, wt, rng = case(n=n, seed=seed, n_vis=1500 + seed)
        y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        V = dev(vis).requires_grad_(True)
        D = autograd.image(V, plan, dev(u), dev(v), dev(w), dev(wt))
        cases.append((u, v, w, vis, wt, y, V))
        outs.append(torch.real(torch.sum(torch.conj(dev(y.astype(np.complex64))) * D[0])))
    for (u, v, w, vis, wt, y, V), loss in zip(cases, outs):  # the first forward's backward first
        loss.backward()
        ref = oracle.degrid(ocfg, u, v, w, vis, y, wt)
        assert rel_err(V.grad.cpu().numpy(), ref) < TOL


def test_kernel_autograd_two_forwards_on_one_plan_before_backward(wst):
    from paper_2301_06061_gb300 import autograd

    n, W = 128, 8
    L = W * 32 + 1
    xs = np.linspace(-W / 2, W / 2, L)
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-200.0, w_max=200.0, support=W, kernel=wst.WST_KERNEL_TABLE,
                     ktable_len=L, kparam=0.0)
    plan = wst.Plan(cfg)
    cases, outs = [], []
    for seed, wiggle in ((31, 0.05), (32, -0.08)):
        u, v, w, vis, wt, rng = case(n=n, n_vis=1200, seed=seed)
        tab = (np.exp(-xs**2 / (2 * 0.925**2)) * (1 + wiggle * np.sin(xs))).astype(np.float32)
        T = dev(tab).requires_grad_(True)
        U = autograd.kernel_image(T, plan, dev(u), dev(v), dev(w), dev(vis), dev(wt))
        dU = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
        cases.append((u, v, w, vis, wt, tab, dU, T))
        outs.append(torch.real(torch.sum(torch.conj(dev(dU)) * U[0])))
    for (u, v, w, vis, wt, tab, dU, T), loss in zip(cases, outs):
        loss.backward()
        ocfg = OracleConfig(n, 0.1, 3, -200.0, 200.0, W, "table", 0.0, tab.astype(np.float64))
        ref = oracle.kernel_grad(ocfg, u, v, w, vis, dU, wt)
        assert np.abs(T.grad.cpu().numpy() - ref).max() < 1e-4 * np.abs(ref).max()


def test_degrid_matches_fp64_central_differences_of_the_oracle_image(wst):
    """wst_degrid against central differences (eps = 1e-3) of the FP64 oracle's image on
    the tiny workload's geometry (256^2, FoV 0.1, 8 planes over [-200, 200], Gaussian
    W = 7).  The image is linear in the visibilities, so the differences are the exact
    derivatives up to FP64 rounding: for L(V) = Re sum conj(y) D(V), dL/dRe V_j =
    Re (A^H y)_j and dL/dIm V_j = Im (A^H y)_j."""
    n, n_w, fov, eps = 256, 8, 0.1, 1e-3
    u, v, w, vis, wt, rng = case(n=n, n_vis=2000, seed=41, fov=fov)
    ocfg = OracleConfig(n, fov, n_w, -200.0, 200.0, 7)
    y = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))

    def loss(values):
        return float(np.real(np.vdot(y, oracle.image(ocfg, u, v, w, values, wt))))

    picks = rng.choice(2000, 12, replace=False)
    fd = np.zeros(picks.size, np.complex128)
    for i, j in enumerate(picks):
        parts = []
        for direction in (1.0, 1j):
            # the oracle reads complex64 values: the step is what V_j +/- eps round to
            lp, lm = vis.copy(), vis.copy()
            lp[j] = np.complex64(np.complex128(vis[j]) + direction * eps)
            lm[j] = np.complex64(np.complex128(vis[j]) - direction * eps)
            step = ((np.complex128(lp[j]) - np.complex128(lm[j])) / direction).real
            parts.append((loss(lp) - loss(lm)) / step)
        fd[i] = parts[0] + 1j * parts[1]
    # the oracle's own adjoint agrees with its differences (FP64 rounding of L / eps)
    ref = oracle.degrid(ocfg, u, v, w, vis, y, wt)[picks]
    assert np.abs(fd - ref).max() < 1e-7 * np.abs(ref).max()
    plan = wst.Plan(wst.Config(n=n, fov=fov, n_w=n_w, w_min=-200.0, w_max=200.0))
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis), dev(wt))
    got = plan.degrid(dev(y.astype(np.complex64)[None])).cpu().numpy()[picks].astype(np.complex128)
    assert np.abs(got - fd).max() < TOL * np.abs(fd).max()


@pytest.mark.parametrize("n,chunk,correct", [(256, 0, True), (256, 2, False), (4096, 0, True)])
def test_degrid_on_the_oversampled_grid_matches_oracle(wst, n, chunk, correct):
    """wst_degrid of a plan with oversample = 2 (grid 2N): the image enters zero-padded
    into the grid (the adjoint of the forward crop), against oracle.degrid_oversampled."""
    u, v, w, vis, wt, rng = case(n=n, seed=50 + n, n_vis=3000)
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-200.0, w_max=200.0, planes_per_chunk=chunk, oversample=2)
    plan = wst.Plan(cfg)
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis), dev(wt))
    y = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    flags = 0 if correct else wst.WST_NO_CORRECTION
    got = plan.degrid(dev(y[None]), flags=flags).cpu().numpy()
    ref = oracle.degrid_oversampled(OracleConfig(n, 0.1, 3, -200.0, 200.0, 7), 2, u, v, w, vis, y, wt,
                                    correct=correct)
    assert rel_err(got, ref) < TOL
    # and the GPU's own dot-product identity with its forward image
    ax = plan.image(flags=flags)[0].cpu().numpy().astype(np.complex128)
    lhs = np.vdot(y.astype(np.complex128), ax)
    rhs = np.vdot(got.astype(np.complex128), vis.astype(np.complex128))
    assert abs(lhs - rhs) < (1e-5 if not correct else 1e-4) * abs(lhs)


def test_table_kernel_and_its_gradient_on_the_oversampled_grid(wst):
    n, W = 256, 8
    L = W * 32 + 1
    u, v, w, vis, wt, rng = case(n=n, n_vis=1500, seed=61)
    xs = np.linspace(-W / 2, W / 2, L)
    tab = (np.exp(-xs**2 / (2 * 0.925**2)) * (1 + 0.05 * np.sin(xs))).astype(np.float32)
    cfg = wst.Config(n=n, fov=0.1, n_w=3, w_min=-200.0, w_max=200.0, support=W, kernel=wst.WST_KERNEL_TABLE,
                     ktable_len=L, kparam=0.0, planes_per_chunk=2, oversample=2)
    plan = wst.Plan(cfg)
    plan.set_kernel_table(dev(tab))
    plan.set_vis(dev(u), dev(v), dev(w), dev(vis), dev(wt))
    ocfg = OracleConfig(n, 0.1, 3, -200.0, 200.0, W, "table", 0.0, tab.astype(np.float64))
    img = plan.image(flags=wst.WST_NO_CORRECTION)[0].cpu().numpy()
    assert rel_err(img, oracle.image_oversampled(ocfg, 2, u, v, w, vis, wt, correct=False)) < TOL
    img_c = plan.image()[0].cpu().numpy()
    assert rel_err(img_c, oracle.image_oversampled(ocfg, 2, u, v, w, vis, wt)) < TOL
    dU = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))).astype(np.complex64)
    got = plan.kernel_grad(dev(dU[None])).cpu().numpy()
    ref = oracle.kernel_grad_oversampled(ocfg, 2, u, v, w, vis, dU, wt)
    assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()
