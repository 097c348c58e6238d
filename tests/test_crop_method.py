"""The full-size GPU tests recompute sampled cells with the oracle on a crop around each cell. This
checks that method on the CPU: crop results equal the full-domain oracle at the crop centre."""
import numpy as np
import pytest

from paper_2506_21804_gb300 import inputs as I
from tests.helpers import oracle_from
from tests.test_gpu_parity import _crop_oracle


@pytest.mark.parametrize("which", ["channel", "canopy", "channel_hrr", "canopy_hrr"])
def test_crop_reproduces_full_domain(which):
    if which.startswith("channel"):
        w = I.channel(nx=24, ny=22, nz=20, seed=3, dtype=np.float64)
        steps, R = (4, 7) if which == "channel" else (3, 7)
    else:
        w = I.canopy(nx=48, ny=30, nz=24, n_buildings=8, seed=2506, domain=(200, 30, 64), crop=(64, 0, 0),
                     dtype=np.float64)
        steps, R = (2, 5) if which == "canopy" else (2, 6)
    if which.endswith("hrr"):
        w.model, w.sigma = 1, 0.5
    full = oracle_from(w)
    full.step(steps)
    rf, uf = full.moments()
    kind = full.classification()[0]
    rng = np.random.default_rng(0)
    picks = list(rng.choice(np.nonzero(kind == 0)[0], 6, replace=False))
    picks += list(rng.choice(np.nonzero(kind == 2)[0], 6, replace=False))
    if (kind == 3).any():
        picks += list(rng.choice(np.nonzero((kind == 3) | (kind == 4))[0], 4, replace=False))
    for n in picks:
        c = (n % w.nx, (n // w.nx) % w.ny, n // (w.nx * w.ny))
        sub, ln = _crop_oracle(w, c, R)
        o = oracle_from(sub)
        o.step(steps)
        ro, uo = o.moments()
        assert abs(ro[ln] - rf[n]) < 1e-14 and np.abs(uo[:, ln] - uf[:, n]).max() < 1e-14, (n, c)
