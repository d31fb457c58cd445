"""Block layout of the two-scale features (§III-C) used by the synthetic-gradient model:
brute-force element loops on CPU tensors."""
import pytest

torch = pytest.importorskip("torch")
from paper_2104_12282_gb300 import onsg  # noqa: E402


def test_block_features_and_targets_match_element_loops():
    nb, (cx, cy, cz) = 2, (3, 2, 2)
    nx, ny, nz = nb * cx, nb * cy, nb * cz
    z = torch.arange(nx * ny * nz, dtype=torch.float64)
    nnc = (cx + 1) * (cy + 1) * (cz + 1)
    uc = torch.arange(3 * nnc, dtype=torch.float64) + 1000.0
    F = onsg.block_features(z, (nx, ny, nz), nb, uc, (cx, cy, cz))
    assert F.shape == (cx * cy * cz, nb ** 3 + 24)
    for K in range(cz):
        for J in range(cy):
            for I in range(cx):
                b = I + cx * (J + cy * K)
                q = 0
                for kk in range(nb):
                    for jj in range(nb):
                        for ii in range(nb):
                            e = (I * nb + ii) + nx * ((J * nb + jj) + ny * (K * nb + kk))
                            assert F[b, q] == z[e]
                            q += 1
                for s in range(8):
                    n = (I + (s & 1)) + (cx + 1) * ((J + ((s >> 1) & 1)) + (cy + 1) * (K + (s >> 2)))
                    for c in range(3):
                        assert F[b, nb ** 3 + 3 * s + c] == uc[c * nnc + n]
    G = onsg.block_gradient(z, (nx, ny, nz), nb, (cx, cy, cz))
    assert torch.equal(G, F[:, :nb ** 3])
    assert torch.equal(onsg.scatter_blocks(G, (nx, ny, nz), nb, (cx, cy, cz)), z)


def test_model_size_matches_table3():
    """125 block values + 24 coarse displacements in, 125 out, 4 x 1000 hidden: 3.3M."""
    m = onsg.make_model(125 + 24, 125)
    n = sum(p.numel() for p in m.parameters())
    assert round(n / 1e6, 1) == 3.3
