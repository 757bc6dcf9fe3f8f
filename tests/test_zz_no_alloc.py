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

    # the configuration is checked before the buffers, so null buffers suffice: a grid of
    # 2^23 columns needs far more than the static scratch's 4096 CTAs for any strip width
    # (PPL_E_NOMEM, not the PPL_E_INVAL of the null pointers), and per-boundary-node arrays
    # would need device copies
    cfg = W.base_config(1 << 23, 4)
    assert ppl.step_noalloc(cfg, 0, 0, 0, 0, 0, 0, 0) == ppl.PPL_E_NOMEM
    cfg = W.base_config(64, 16, hydro_bc=[W.PERIODIC, W.PERIODIC, W.WALL, W.WALL],
                        rho_w=[None, None, np.ones(64), None])
    assert ppl.step_noalloc(cfg, 0, 0, 0, 0, 0, 0, 0) == ppl.PPL_E_INVAL


def test_step_noalloc_rejects_misaligned_and_overlapping_buffers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04560_gb300 import ppl

    cfg = W.base_config(64, 16)
    n = 64 * 16
    buf = torch.zeros(2 * 10 * n + 16, dtype=torch.float64, device="cuda")
    p = buf.data_ptr()
    fi, ti, fo, to = p, p + 9 * n * 8, p + 10 * n * 8, p + 19 * n * 8
    st = torch.zeros(4, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    args = (st.data_ptr(), st.data_ptr() + 8, status.data_ptr())
    # misaligned state pointers and outputs overlapping an input are refused before any launch
    assert ppl.step_noalloc(cfg, fi + 4, ti, fo, to, *args) == ppl.PPL_E_INVAL
    assert ppl.step_noalloc(cfg, fi, ti, fo, to + 4, *args) == ppl.PPL_E_INVAL
    assert ppl.step_noalloc(cfg, fi, ti, fi + 8 * n, to, *args) == ppl.PPL_E_INVAL
    assert ppl.step_noalloc(cfg, fi, ti, fo, ti + 8, *args) == ppl.PPL_E_INVAL
    assert ppl.step_noalloc(cfg, fi, ti, fo, fo + 8 * 8 * n, *args) == ppl.PPL_E_INVAL


def _raw_state(sim, path, np_dtype):
    """The handle's stored state as the step kernel sees it (checkpoint file: a 48-byte header,
    rho_bar and mass as two doubles, then f [9][ny][nx] and T [ny][nx] in the working precision)."""
    sim.save(str(path))
    raw = np.fromfile(str(path), dtype=np.uint8)
    n = sim.nx * sim.ny
    stats = raw[48:64].view(np.float64).copy()
    body = raw[64:].view(np_dtype)
    return body[:9 * n].reshape(9, sim.ny, sim.nx).copy(), body[9 * n:].reshape(sim.ny, sim.nx).copy(), stats


def test_step_noalloc_fp32_matches_ppl_step_twice(tmp_path):
    # FP32 deviation storage on an x-periodic grid with even nx: the two-column kernel, staging
    # rows with per-thread copies here and with tensor copies on the handle
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2201_04560_gb300 import Simulation, ppl

    a, b, R, om = 3 / 49, 2 / 21, 1.0, 0.344
    Tc = ppl.tc(a, b, R)
    rv, rl, _ = ppl.maxwell(a, b, R, om, 0.8 * Tc)
    cfg, ic = W.droplet_vaporization(Tc, rv, rl, 0.1, nx=256, ny=72, R0=20.0, iso_steps=0, precision="fp32")
    sim = Simulation(cfg, *ic)
    assert sim.kernel == "pair"
    sim.step(5)
    f0, T0, st0 = _raw_state(sim, tmp_path / "a.bin", np.float32)
    fa = torch.from_numpy(f0).cuda().contiguous()
    Ta = torch.from_numpy(T0).cuda().contiguous()
    fb, Tb = torch.empty_like(fa), torch.empty_like(Ta)
    s0 = torch.tensor([st0[0]], dtype=torch.float64, device="cuda")
    s1 = torch.zeros(2, dtype=torch.float64, device="cuda")
    s2 = torch.zeros(2, dtype=torch.float64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert ppl.step_noalloc(cfg, fa.data_ptr(), Ta.data_ptr(), fb.data_ptr(), Tb.data_ptr(), s0.data_ptr(),
                            s1.data_ptr(), status.data_ptr()) == 0
    assert ppl.step_noalloc(cfg, fb.data_ptr(), Tb.data_ptr(), fa.data_ptr(), Ta.data_ptr(), s1.data_ptr(),
                            s2.data_ptr(), status.data_ptr()) == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    sim.step(2)
    f2, T2, st2 = _raw_state(sim, tmp_path / "b.bin", np.float32)
    sim.close()
    # same arithmetic on the same launch shape: the staging path only moves data
    np.testing.assert_allclose(fa.cpu().numpy(), f2, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(Ta.cpu().numpy(), T2, rtol=1e-6, atol=1e-9)
    assert float(s2[0].item()) == pytest.approx(st2[0], rel=1e-12)
    assert float(s2[1].item()) == pytest.approx(st2[1], rel=1e-12)
