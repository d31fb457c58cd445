"""An OC run stopped at a checkpoint and resumed follows the uninterrupted run: the same
compliance history to the solver's tolerance (the resumed first solve starts from zero
instead of the previous displacement) and the same final design to 1e-4."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_2104_12282_gb300 import optimize as O  # noqa: E402
from paper_2104_12282_gb300 import problems as P  # noqa: E402


def test_resumed_run_follows_the_uninterrupted_run(tmp_path):
    p = P.cantilever(24, 12, 12, volfrac=0.3, rmin=1.5)
    z_full, h_full = O.run(p, 12, rtol=1e-8)
    ck = str(tmp_path / "oc.npz")
    O.run(p, 6, rtol=1e-8, checkpoint=ck, checkpoint_every=3)
    k, _, h_mid, _ = O.load_checkpoint(ck)
    assert k == 6 and len(h_mid) == 6
    z_res, h_res = O.run(p, 12, rtol=1e-8, checkpoint=ck, resume=True)
    assert [r["it"] for r in h_res] == list(range(12))
    c_full = np.array([r["c"] for r in h_full])
    c_res = np.array([r["c"] for r in h_res])
    assert np.abs(c_res / c_full - 1.0).max() <= 1e-5
    assert torch.max(torch.abs(z_res - z_full)).item() <= 1e-4
