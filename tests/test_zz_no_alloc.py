"""The allocation-free step entry point (ppl_step_noalloc), for callers that cannot call
cudaMalloc: two calls in a row through the C ABI must reproduce two steps of the
handle-based ppl_step on the same state. Collected last on purpose."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-10


def test_step_noalloc_matches_ppl_step_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04560_gb300 import Simulation, ppl

    a, b, R, om = 3 / 49, 2 / 21, 1.0, 0.344
    Tc = ppl.tc(a, b, R)
    rv, rl, _ = ppl.maxwell(a, b, R, om, 0.86 * Tc)
    # walls, outflow and the energy equation, scalar (per-side) boundary values only
    cfg, ic = W.stefan_strip(Tc, rv, rl, 0.1032, nx=203, ny=37, n_vapour=10)
    ny, nx = cfg["ny"], cfg["nx"]
    sim = Simulation(cfg, *ic)
    sim.step(3)
    f0 = torch.from_numpy(sim.populations()).cuda().contiguous()
    T0 = torch.from_numpy(sim.fields()["T"]).cuda().contiguous()
    n0 = sim.norms()
    f1, T1 = torch.empty_like(f0), torch.empty_like(T0)
    st0 = torch.tensor([n0["rho_mean"]], dtype=torch.float64, device="cuda")
    st1 = torch.zeros(2, dtype=torch.float64, device="cuda")
    st2 = torch.zeros(2, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")

    rc = ppl.step_noalloc(cfg, f0.data_ptr(), T0.data_ptr(), f1.data_ptr(), T1.data_ptr(), st0.data_ptr(),
                          st1.data_ptr(), status.data_ptr())
    assert rc == 0, rc
    rc = ppl.step_noalloc(cfg, f1.data_ptr(), T1.data_ptr(), f0.data_ptr(), T0.data_ptr(), st1.data_ptr(),
                          st2.data_ptr(), status.data_ptr())
    assert rc == 0, rc
    torch.cuda.synchronize()
    assert int(status.item()) == 0

    sim.step(2)
    want_f = sim.populations()
    want_T = sim.fields()["T"]
    n2 = sim.norms()
    sim.close()
    got_f = f0.cpu().numpy()
    got_T = T0.cpu().numpy()
    inner = slice(0, nx - 1)  # the outflow column is an implicit copy, never stored by a step
    np.testing.assert_allclose(got_f[:, :, inner], want_f[:, :, inner], rtol=FP64_RTOL, atol=1e-13)
    np.testing.assert_allclose(got_T[:, inner], want_T[:, inner], rtol=FP64_RTOL, atol=0)
    assert float(st2[1].item()) == pytest.approx(n2["mass"], rel=1e-12)


def test_step_noalloc_rejects_what_it_cannot_hold():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04560_gb300 import ppl

    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    # a grid wider than the static scratch's 4096 column strips
    cfg = W.base_config(4096 * 122 + 1, 4)
    assert ppl.step_noalloc(cfg, p, p + 8, p + 16, p + 24, p, p, p) == ppl.PPL_E_INVAL
    # per-boundary-node arrays would need device copies
    cfg = W.base_config(64, 16, hydro_bc=[W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                        rho_w=[None, None, np.ones(64), None])
    assert ppl.step_noalloc(cfg, p, p + 8, p + 16, p + 24, p, p, p) == ppl.PPL_E_INVAL
