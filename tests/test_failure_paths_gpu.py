"""Failure paths of the library, driven by host-side inputs only (no kernel is made to fail).

* a Krylov cap that is too small: STDG_ENOTCONV, filled statistics, the state, time and
  receiver records still advanced;
* non-finite inputs on a live context: STDG_EINVAL, and the context keeps working;
* an input that overflows: the residual sentinel stops the solve at once with
  STDG_ENONFINITE instead of iterating to the cap;
* the device error word of the face kernel's bounded bulk-copy waits, set from the host:
  reported once as STDG_ECUDA by the next checking call, then cleared;
* the energy-growth sentinel (Theorem 4): silent on source-free steps, which dissipate
  (space-time DG) or keep (Crank-Nicolson) the energy; tripped by a tolerance that demands
  a decrease no step gives (a host-side setting), with the state advanced; skipped when
  sources drive the solution.
"""
import numpy as np
import pytest

import synth
from helpers import gpu_solver, need_gpu, rel_l2

pytestmark = pytest.mark.gpu


def _small(p=2):
    return synth.scaled("c2", ny=6, p=p, steps=2)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_max_iters_cap_reports_notconv_and_advances_the_state(precision):
    need_gpu()
    from paper_1802_04516_gb300.binding import STDG_ENOTCONV
    w = _small()
    s = gpu_solver(w, precision=precision, rel_tol=1e-13, max_iters=3)
    v0, _ = s.get_state()
    st = s.step(w.dt, 2, allow_notconv=True)
    assert st["status"] == STDG_ENOTCONV
    assert st["iters_max"] > 0
    assert st["iters_total"] >= st["iters_max"]
    assert st["final_rel_res"] > 1e-13
    assert abs(s.time - 2 * w.dt) < 1e-15
    assert s.read_receivers().shape[1] == 2
    v1, _ = s.get_state()
    assert np.isfinite(v1).all() and np.abs(v1 - v0).max() > 0
    # the same context converges with a sensible cap afterwards
    s2 = gpu_solver(w, precision=precision, rel_tol=1e-10, max_iters=20000)
    assert s2.step(w.dt, 1)["status"] == 0


def test_non_finite_inputs_are_rejected_on_a_live_context():
    need_gpu()
    from paper_1802_04516_gb300.binding import STDG_EINVAL, StdgError
    w = _small()
    s = gpu_solver(w, rel_tol=1e-10, max_iters=20000)
    s.step(w.dt, 1)
    v, sig = s.get_state()
    bad = []
    lam = w.lam.copy()
    lam[3] = np.nan
    bad.append(lambda: s.set_material(lam, w.mu, w.rho))
    rho = w.rho.copy()
    rho[0] = np.inf
    bad.append(lambda: s.set_material(w.lam, w.mu, rho))
    vb = v.copy()
    vb.flat[7] = np.inf
    bad.append(lambda: s.set_state(vb, sig))
    sb = sig.copy()
    sb.flat[11] = np.nan
    bad.append(lambda: s.set_state(v, sb))
    xs = np.array(w.shots_xs, dtype=float)
    xs[0, 0] = np.nan
    bad.append(lambda: s.set_sources(xs, w.shots_dir, w.f0, w.t_delay, w.a1))
    bad.append(lambda: s.set_sources(w.shots_xs, w.shots_dir, np.nan, w.t_delay, w.a1))
    xr = np.array(w.receivers, dtype=float)
    xr[2, 1] = np.inf
    bad.append(lambda: s.set_receivers(xr))
    for k, call in enumerate(bad):
        with pytest.raises(StdgError) as ei:
            call()
        assert ei.value.code == STDG_EINVAL, k
    # nothing was taken over: the context steps on from the state it had
    v_before, _ = s.get_state()
    assert rel_l2(v_before, v) == 0.0
    assert s.step(w.dt, 1)["status"] == 0


def test_overflowing_source_stops_the_solve_with_nonfinite():
    need_gpu()
    from paper_1802_04516_gb300.binding import STDG_ENONFINITE, StdgError
    w = _small()
    for precision in ("fp64", "mixed"):
        s = gpu_solver(w, precision=precision, rel_tol=1e-10, max_iters=5000)
        s.set_sources(w.shots_xs, w.shots_dir, w.f0, 0.0, 1e305)   # finite amplitude; the slab's b overflows
        with pytest.raises(StdgError) as ei:
            s.step(w.dt, 1)
        assert ei.value.code == STDG_ENONFINITE
        assert s.last_stats["status"] == STDG_ENONFINITE
        assert s.last_stats["iters_max"] < 50          # stopped at once, not at the cap


def test_bounded_wait_error_is_reported_once_and_cleared():
    torch = need_gpu()
    from paper_1802_04516_gb300.binding import STDG_ECUDA, StdgError
    w = _small(p=3)
    s = gpu_solver(w, precision="mixed", rel_tol=1e-10, max_iters=20000)
    s.step(w.dt, 1)
    s.inject_wait_error()
    with pytest.raises(StdgError) as ei:
        s.step(w.dt, 1)
    assert ei.value.code == STDG_ECUDA and "wait gave up" in str(ei.value)
    assert abs(s.time - 2 * w.dt) < 1e-15            # the graph ran: time and records advanced
    assert s.read_receivers().shape[1] == 2
    assert s.step(w.dt, 1)["status"] == 0            # reported once, then cleared
    # the FP32 operator on caller buffers checks the word too
    n = s.nvel
    x = torch.randn(n, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    s.inject_wait_error()
    with pytest.raises(StdgError) as ei:
        s.apply_operator_device(w.dt, x.data_ptr(), y.data_ptr(), fp32=True)
    assert ei.value.code == STDG_ECUDA
    y.zero_()
    s.apply_operator_device(w.dt, x.data_ptr(), y.data_ptr(), fp32=True)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all() and float(y.abs().max()) > 0


def _periodic(scheme, precision, p):
    from paper_1802_04516_gb300.binding import Solver
    xyz, ev, per = synth.tri_grid(6, 6, 1.0, 1.0, periodic=True, jitter=0.2, seed=21)
    pg = 0 if scheme == "cn" else p
    s = Solver(2, p, pg, scheme, precision, rel_tol=1e-12 if precision == "fp64" else 1e-9, max_iters=5000,
               gmres_restart=30, preconditioner=1)
    s.set_mesh(xyz, ev, per)
    s.set_material(*synth.homogeneous(ev.shape[0], 2.0, 1.0, 1.0))
    s.set_shots(1)
    s.set_plane_wave(0, [1.0, 0.0], amp=0.01)
    return s


@pytest.mark.parametrize("scheme,precision,tol", [("stdg", "fp64", 1e-12), ("stdg", "mixed", 1e-8),
                                                  ("cn", "fp64", 1e-10)])
def test_energy_sentinel_is_silent_on_source_free_steps(scheme, precision, tol):
    need_gpu()
    s = _periodic(scheme, precision, 2)
    s.set_energy_check(True, tol)
    e0 = s.energy()[0]
    for _ in range(3):
        st = s.step(0.02, 2)
        assert st["status"] == 0
    e1 = s.energy()[0]
    assert 0 < e1 <= (1 + tol) * e0


def test_energy_sentinel_trips_on_a_demanded_decrease_and_advances_the_state():
    from paper_1802_04516_gb300.binding import STDG_EENERGY, StdgError
    need_gpu()
    s = _periodic("stdg", "fp64", 2)
    e0 = s.energy()[0]
    s.set_energy_check(True, -0.5)   # demands that each call halve the energy: no step does
    with pytest.raises(StdgError) as ei:
        s.step(0.02, 1)
    assert ei.value.code == STDG_EENERGY and "grew" in str(ei.value)
    assert abs(s.time - 0.02) < 1e-15        # the step ran and the state advanced
    e1 = s.energy()[0]
    assert 0.5 * e0 < e1 <= e0 * (1 + 1e-12)
    s.set_energy_check(False)
    assert s.step(0.02, 1)["status"] == 0
    with pytest.raises(StdgError):
        s.set_energy_check(True, -1.0)       # rel_tol must be > -1


def test_energy_sentinel_is_skipped_when_sources_drive_the_solution():
    need_gpu()
    w = _small()
    s = gpu_solver(w, precision="fp64", rel_tol=1e-12, max_iters=5000)
    s.set_energy_check(True, -0.5)           # would trip on any source-free step
    assert s.step(w.dt, 2)["status"] == 0
