"""The OC run's checkpoint file (optimize.save_checkpoint / load_checkpoint) on the CPU:
round trip of the design, history and smoother, and no partial file left behind."""
import os

import numpy as np

from paper_2104_12282_gb300 import optimize as O


def test_checkpoint_round_trip(tmp_path):
    path = str(tmp_path / "run.npz")
    z = np.random.default_rng(0).uniform(0, 1, 1000).astype(np.float32)
    hist = [{"it": 0, "c": 12.5, "change": 0.2}, {"it": 1, "c": 11.0, "change": 0.15}]
    O.save_checkpoint(path, 2, z, hist, (1, 3))
    k, z2, h2, sm = O.load_checkpoint(path)
    assert k == 2 and sm == (1, 3) and h2 == hist
    assert z2.dtype == np.float32 and np.array_equal(z2, z)
    assert sorted(os.listdir(tmp_path)) == ["run.npz"]   # the temporary file was renamed
    O.save_checkpoint(path, 3, z[::-1].copy(), hist + [{"it": 2}], (2, 2))   # overwrite
    k, z3, h3, sm = O.load_checkpoint(path)
    assert k == 3 and sm == (2, 2) and len(h3) == 3 and np.array_equal(z3, z[::-1])
    # the full setting: degrees, interval ratio, bound and W-cycle mask
    O.save_checkpoint(path, 4, z, hist, (1, 3, 30.0, 3.6163636363636376, 2))
    k, _, _, sm = O.load_checkpoint(path)
    assert k == 4 and sm == (1, 3, 30.0, 3.6163636363636376, 2)
    assert isinstance(sm[0], int) and isinstance(sm[4], int)
