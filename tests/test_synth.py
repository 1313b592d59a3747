"""The seeded input generator: the device-side orbital builder agrees with the
NumPy one, and the MD-like drift is reproducible."""
import numpy as np

from paper_1911_10630_gb300 import synth


def test_orbitals_torch_matches_numpy():
    torch = __import__("torch")
    w = synth.tiny(seed=2, n=5, npts=20, length=6.0)
    a = w.orbitals()
    b = synth.orbitals_torch(w, device="cpu", chunk=2).numpy()
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
    assert torch.float64 == torch.float64


def test_md_drift_is_cumulative_and_seeded():
    w1 = synth.config4(0, 1)
    w2 = synth.config4(0, 2)
    again = synth.config4(0, 2)
    assert np.array_equal(w2.centers, again.centers)
    step = synth.config4(0, 0).centers
    d1 = w1.centers - step
    d1 -= w1.cell * np.round(d1 / w1.cell)
    assert 0.005 < np.std(d1) < 0.04  # one N(0, 0.02^2) draw per component
    assert w1.n == 1024 and int(w1.grid[0]) == 190
