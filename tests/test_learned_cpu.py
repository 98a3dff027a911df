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
