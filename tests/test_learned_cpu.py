"""Host-side pieces of the learned kernel, against the oracle (CPU only)."""
import numpy as np

import oracle
from oracle import OracleConfig


def test_correction_matrix_is_the_table_transform():
    from paper_2301_06061_gb300 import learned

    n, W, per = 64, 8, 128  # 3-point rule per interval: truncation ~ (1/per)^6
    L = W * per + 1
    rng = np.random.default_rng(3)
    tab = np.exp(-np.linspace(-4, 4, L) ** 2 / 1.7) * (1 + 0.2 * rng.random(L))
    M = learned.correction_matrix(n, W, L)
    cfg = OracleConfig(n, 0.1, 1, 0.0, 0.0, W, "table", 0.0, tab)
    ref = oracle.kernel_ft(cfg, (np.arange(n) - n // 2) / n)
    np.testing.assert_allclose(M @ tab, ref, rtol=1e-11, atol=1e-13)


def test_mlp_kernel_is_even_and_tabulated_on_the_support():
    import torch

    from paper_2301_06061_gb300 import learned

    torch.manual_seed(0)
    mlp = learned.KernelMLP(8)
    x = torch.linspace(-4, 4, 101)
    assert torch.allclose(mlp(x), mlp(-x))
    tab = learned.tabulate(mlp, 8, per_cell=4)
    assert tab.shape == (33,)
    assert torch.allclose(tab, torch.flip(tab, [0]))


def _cpu_trainer(learned):
    """A Trainer whose sky and loss are host stand-ins (no plan, no GPU): the training
    loop, the optimiser and the checkpoint logic are the real ones."""
    import torch

    tr = object.__new__(learned.Trainer)
    tr.support, tr.per_cell, tr.device = 8, 16, torch.device("cpu")
    tr.sky_case = lambda i: i
    tr.loss = lambda table, i: ((table - 0.01 * (i % 5)) ** 2).mean()
    return tr


def test_training_resumes_from_a_checkpoint_as_if_uninterrupted(tmp_path):
    """Six steps in one go against four steps (checkpoints at 2 and 4), then a fresh model
    and optimiser resumed from the checkpoint for the last two: the losses and the final
    parameters agree exactly."""
    import torch

    from paper_2301_06061_gb300 import learned

    tr = _cpu_trainer(learned)
    torch.manual_seed(5)
    ref = learned.KernelMLP(8)
    ref_hist = tr.train(ref, range(6), lr=1e-2)

    ckpt = str(tmp_path / "train.pt")
    torch.manual_seed(5)
    first = learned.KernelMLP(8)
    tr.train(first, range(4), lr=1e-2, checkpoint=ckpt, checkpoint_every=2)
    torch.manual_seed(99)  # a different initialisation: everything must come from the file
    resumed = learned.KernelMLP(8)
    hist = tr.train(resumed, range(6), lr=1e-2, checkpoint=ckpt, checkpoint_every=2)

    assert hist == ref_hist
    for a, b in zip(ref.state_dict().values(), resumed.state_dict().values()):
        assert torch.equal(a, b)
    step, saved = learned.load_checkpoint(ckpt, learned.KernelMLP(8),
                                          torch.optim.Adam(learned.KernelMLP(8).parameters()))
    assert step == 6 and saved == ref_hist
    assert not (tmp_path / "train.pt.tmp").exists()


def test_trained_kernel_tabulated_at_any_resolution():
    """The stored table is the network at 1024 samples per cell; table_at resamples the
    network (the bench grids with 128 per cell, whose tap table stays in L1)."""
    import os

    from paper_2301_06061_gb300 import learned

    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2301_06061_gb300",
                        "data", "learned_kernel_w8.npz")
    stored = learned.load_table(path)
    again = learned.table_at(path, 1024)
    assert np.array_equal(stored, again)
    coarse = learned.table_at(path, 128)
    assert coarse.size == 8 * 128 + 1
    # every 8th sample of the fine table is a sample of the coarse one (the same nodes)
    assert np.abs(coarse - stored[::8]).max() < 1e-6
