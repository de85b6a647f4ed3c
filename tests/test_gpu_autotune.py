"""pdg_mc_autotune: the library's own sweep over (PIPG form, CTA size)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_autotune_picks_and_applies_a_candidate(inputs):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_18034_gb300 import build
    from paper_2404_18034_gb300.autotune import candidates
    from paper_2404_18034_gb300.pdg_mc import Solver
    build.build()
    p = inputs.load_params()
    x0 = torch.from_numpy(inputs.dispersion(p, 64, 3, "bj")).cuda()
    for prec in (0, 1):
        S = Solver(p, 10, prec)
        t, f, rate = S.autotune(x0, None, 1)
        assert (f, t) in candidates(10, 4, prec) and rate > 0
        out = S.solve(x0, mode=1)
        torch.cuda.synchronize()
        info = S.launch_info()
        assert info["threads"] == t and info["pipg_form"] == f
        assert np.mean(out["status"].cpu().numpy() == 0) > 0.5
        S.close()
