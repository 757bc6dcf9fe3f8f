"""GPU: the refinement-study drivers (refinement.py) on small meshes and short runs — they
complete, return finite measures of the right shape, and keep their bookkeeping (substeps
per mesh, time-shift window) consistent. The full-size studies are bench.py experiments."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04560_gb300 import refinement
    return refinement


def test_substeps_follow_dt_dx2(R):
    assert R.substeps([128, 256, 512], 128) == [1, 4, 16]
    assert R.substeps([160, 240, 360, 540], 160) == [64, 144, 324, 729]


def test_droplet_vaporization_study_small(R):
    out = R.droplet_vaporization_study(meshes=(32, 64), R0=8.0, iso_steps=100, coarse_steps=600, sample_every=50,
                                       autotune_steps=0)
    assert out["substeps"] == [1, 4]
    assert len(out["R"][0]) == len(out["R"][1]) == len(out["t"]) == 12
    assert all(math.isfinite(r) and 4.0 < r < 12.0 for series in out["R"] for r in series)
    assert 0.0 <= out["delta_R"][0] < 0.2


def test_contact_and_gw_studies_small(R):
    import workloads as W
    out = R.contact_angle_study(meshes=(40, 60), value=2.3, coarse_steps=800, autotune_steps=0)
    assert len(out["theta"]) == 2 and all(0.0 <= t <= 180.0 for t in out["theta"] if not math.isnan(t))
    assert len(out["delta_rho"]) == 1 and 0.0 <= out["delta_rho"][0] < 0.5
    g = R.G_w_search(meshes=(40, 60), coarse_steps=800, max_iter=4, tol=2.0)
    assert g["meshes"][0]["G_w"] == -0.8 and len(g["meshes"]) == 2
    assert g["meshes"][1]["evaluations"] <= 4
    assert W.CONTACT_MOD_PSI == 1


def test_pool_boiling_study_small(R):
    out = R.pool_boiling_study(meshes=(80, 120), coarse_steps=640, sample_every=64, tau=320, m=128, shift_stride=64,
                               autotune_steps=0)
    assert out["substeps"] == [4, 9]
    for f in ("rho", "T"):
        assert len(out["d"][f]) == 1 and len(out["d"][f][0]) == len(out["t"]) == 10
        assert 0.0 <= out["D"][f][0] < 1.0
    assert np.all(np.isfinite(np.array(out["Q"])))
    assert len(out["shifts"]) == 1 and abs(out["shifts"][0]["delta"]) <= 128


def test_stefan_study_small(R):
    out = R.stefan_study(param_set=2, meshes=(80, 160), coarse_steps=400, sample_every=40, autotune_steps=0)
    assert out["substeps"] == [1, 4]
    assert len(out["s"][0]) == len(out["s"][1]) == 10
    s0, s1 = np.array(out["s"][0]), np.array(out["s"][1])
    assert np.all(np.isfinite(s0)) and np.all(np.isfinite(s1))
    assert np.all((s0 > 0) & (s0 < 80)) and abs(s0[-1] - s1[-1]) < 3.0
    assert 0.0 <= out["delta_s"][0] < 0.5
