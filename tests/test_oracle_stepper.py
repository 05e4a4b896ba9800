"""Pins of the oracle's time stepping against the paper's theorems and exact solutions."""
import numpy as np
import pytest

import synth
from oracle.stepper import Simulation, ricker


def _run_energy(sim, steps):
    out = [sim.energy()]
    jumps = []
    for _ in range(steps):
        sim.step(1)
        out.append(sim.energy())
        if sim.scheme == "stdg":
            jumps.append(sim.jump_dissipation())
    return np.array(out), np.array(jumps)


def _random_state(sim, seed):
    rng = np.random.default_rng(seed)
    sim.set_state(rng.normal(size=sim.v_tr.shape), rng.normal(size=sim.sig_tr.shape))


@pytest.mark.parametrize("dim,p,periodic,hetero", [(2, 2, True, False), (2, 3, False, True), (3, 2, True, False),
                                                  (3, 1, False, True)])
def test_crank_nicolson_preserves_energy(dim, p, periodic, hetero):
    # Theorem 5 (Eq. SP3F): exact energy preservation, also with free-surface faces
    if dim == 2:
        xyz, ev, per = synth.tri_grid(4, 4, 1.0, 1.0, periodic=periodic, jitter=0.2, seed=7)
    else:
        xyz, ev, per = synth.tet_kuhn(3 if periodic else 2, 1.0, periodic=periodic, jitter=0.1, seed=7)
    n = ev.shape[0]
    rng = np.random.default_rng(2)
    lam, mu, rho = (rng.uniform(1, 3, n), rng.uniform(.5, 1.5, n), rng.uniform(.7, 1.4, n)) if hetero else \
        (np.full(n, 2.0), np.full(n, 1.0), np.full(n, 1.0))
    sim = Simulation(xyz, ev, per, lam, mu, rho, p, 0, "cn", 0.37)
    _random_state(sim, 3)
    e, _ = _run_energy(sim, 4)
    assert np.abs(e / e[0] - 1).max() < 1e-12


@pytest.mark.parametrize("dim,p,pg,periodic", [(2, 1, 1, True), (2, 2, 2, False), (2, 3, 1, True), (3, 1, 1, False),
                                               (3, 2, 2, True)])
def test_space_time_energy_loss_equals_time_jumps(dim, p, pg, periodic):
    # Theorem 4, eq. stsum4: E^{n+1} - E^n + (time-jump terms at t^n) = 0, jumps >= 0
    if dim == 2:
        xyz, ev, per = synth.tri_grid(4, 4, 1.0, 1.0, periodic=periodic, jitter=0.2, seed=8)
    else:
        xyz, ev, per = synth.tet_kuhn(3 if periodic else 2, 1.0, periodic=periodic, jitter=0.1, seed=8)
    n = ev.shape[0]
    rng = np.random.default_rng(4)
    sim = Simulation(xyz, ev, per, rng.uniform(1, 3, n), rng.uniform(.5, 1.5, n), rng.uniform(.7, 1.4, n),
                     p, pg, "stdg", 0.21)
    _random_state(sim, 5)
    e, jumps = _run_energy(sim, 3)
    assert (jumps >= 0).all()
    assert (np.diff(e) <= 1e-14 * e[0]).all()
    np.testing.assert_allclose(e[:-1] - e[1:], jumps, rtol=1e-9, atol=1e-13 * e[0])


def _plane_wave_error(n, p, pg, scheme, periods=1.0, cfl=0.25):
    w = synth.c1_periodic_pwave(n=n, p=p)
    cp = 2.0
    dt = cfl / n / cp
    steps = int(round(periods / cp / dt))
    dt = periods / cp / steps
    sim = Simulation(w.xyz, w.elem_vert, w.period, w.lam, w.mu, w.rho, p, pg, scheme, dt)
    sim.set_plane_wave(0, np.array([1.0, 0.0]), None, 1e-2)
    v0, s0 = sim.v_tr.copy(), sim.sig_tr.copy()
    sim.step(steps)
    # one full period later the exact solution equals the initial one (Sec. 6.2)
    return np.linalg.norm(sim.v_tr - v0) / np.linalg.norm(v0)


@pytest.mark.parametrize("p,pg,scheme,order", [(1, 1, "stdg", 2.0), (2, 2, "stdg", 3.0), (2, 0, "cn", 2.0)])
def test_plane_wave_convergence_order(p, pg, scheme, order):
    # Table tab:NT1: order p+1 for p = p_gamma; Crank-Nicolson is second order in time
    e1 = _plane_wave_error(6, p, pg, scheme)
    e2 = _plane_wave_error(12, p, pg, scheme)
    rate = np.log2(e1 / e2)
    assert rate > order - 0.35, (e1, e2, rate)
    assert e2 < 5e-2


def test_ricker_closed_form():
    f0, td, a1 = 10.0, 0.116, 1.0
    t = np.linspace(0, 0.3, 31)
    ref = 0.5 * a1 * (1 - 2 * (np.pi * f0 * (t - td)) ** 2) * np.exp(-(np.pi * f0 * (t - td)) ** 2)
    np.testing.assert_allclose(ricker(t, f0, td, a1), ref, atol=1e-15)
    assert abs(ricker(td, f0, td, a1) - 0.5 * a1) < 1e-15


def test_source_linearity_and_superposition():
    w = synth.scaled("c2", ny=6, steps=4)
    base = Simulation.from_workload(w)
    src = dict(xs=w.shots_xs[0], direction=w.shots_dir[0], f0=w.f0, t_delay=0.02, a1=1.0)

    def run(ic, a1):
        s = Simulation.from_workload(w)
        if ic:
            _random_state(s, 11)
        if a1 != 0.0:
            s.set_source(**{**src, "a1": a1})
        s.step(4)
        return s.v_tr.copy(), s.sig_tr.copy()

    v_ic, s_ic = run(True, 0.0)
    v_src, s_src = run(False, 1.0)
    v_both, s_both = run(True, 1.0)
    v_two, _ = run(False, 2.0)
    np.testing.assert_allclose(v_both, v_ic + v_src, atol=1e-12 * np.abs(v_both).max())
    np.testing.assert_allclose(s_both, s_ic + s_src, atol=1e-12 * np.abs(s_both).max())
    np.testing.assert_allclose(v_two, 2 * v_src, atol=1e-13 * np.abs(v_two).max())
    assert np.abs(v_src).max() > 0
    del base


def test_receiver_at_node_reads_nodal_value():
    w = synth.c1_periodic_pwave(n=5, p=2)
    sim = Simulation.from_workload(w)
    _random_state(sim, 1)
    # centroid of element 7: evaluate the polynomial directly from the nodal values
    x = sim.mesh.X[7].mean(axis=0)
    sim.set_receivers(x[None])
    val = sim.receiver_values()[0]
    xi = np.linalg.solve(sim.mesh.J[7], x - sim.mesh.X[7, 0])
    phi = sim.disc.ref.values(xi[None])[0]
    np.testing.assert_allclose(val, sim.v_tr[7] @ phi, rtol=1e-13)


@pytest.mark.parametrize("kind,n,pol", [(0, [1.0, 1.0], None), (1, [1.0, 1.0], None), (1, [0.6, -0.8], None),
                                        (0, [1.0, 0.0, 0.0], None), (1, [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]),
                                        (1, [1.0, 2.0, 2.0], [2.0, -1.0, 0.0])])
def test_plane_wave_fields_solve_the_elastic_wave_equations(kind, n, pol):
    # Eqs. NT2.1-NT2.2 (unit normal, reading of the paper's eigenvectors): the exact P and S
    # waves satisfy rho dv/dt = div sigma and dsigma/dt = lam tr(grad v) I + mu (grad v + grad v^T),
    # checked by central differences at random points (Eq. 1 of the velocity-stress system)
    from oracle.stepper import plane_wave_fields
    lam, mu, rho, amp = 2.0, 1.0, 1.3, 0.7
    d = len(n)
    rng = np.random.default_rng(4)
    x = rng.uniform(-1, 1, size=(7, d))
    t, h = 0.37, 1e-5

    def f(xx, tt):
        return plane_wave_fields(xx, tt, kind, n, pol, amp, lam, mu, rho)

    v_t = (f(x, t + h)[0] - f(x, t - h)[0]) / (2 * h)
    s_t = (f(x, t + h)[1] - f(x, t - h)[1]) / (2 * h)
    grad_v = np.zeros((7, d, d))      # [q, k, l] = d v_k / d x_l
    div_s = np.zeros((7, d))
    for l in range(d):
        e = np.zeros(d)
        e[l] = h
        vp, sp = f(x + e, t)
        vm, sm = f(x - e, t)
        grad_v[:, :, l] = (vp - vm) / (2 * h)
        div_s += (sp[:, :, l] - sm[:, :, l]) / (2 * h)
    scale = amp * 2 * np.pi * np.linalg.norm(n) * (lam + 2 * mu)
    assert np.abs(rho * v_t - div_s).max() < 1e-7 * scale
    strain_rate = lam * np.trace(grad_v, axis1=1, axis2=2)[:, None, None] * np.eye(d) + mu * (
        grad_v + np.swapaxes(grad_v, 1, 2))
    assert np.abs(s_t - strain_rate).max() < 1e-7 * scale
    assert np.abs(f(x, t)[0]).max() > 1e-3 * amp                 # not the zero solution


def test_source_vector_is_the_slab_integral_of_the_wavelet():
    # Sec. 6.3 point source: (rho S)_i = d phi(x_s) dt int_0^1 gamma_a(tau) S(t0 + tau dt) dtau in the
    # source element only.  Against an adaptive quadrature of the same integral (scipy) and the
    # partition of unity of the nodal basis (the phi(x_s) sum to 1)
    from scipy.integrate import quad
    w = synth.scaled("c2", ny=6, steps=2)
    sim = Simulation.from_workload(w)
    sim.set_source(w.shots_xs[0], w.shots_dir[0], w.f0, w.t_delay, w.a1)
    dz = sim.disc
    e_s = sim.sources["elem"]
    for t0 in (0.5 * w.t_delay, w.t_delay - 0.3 * sim.dt, 1.7 * w.t_delay):
        sv = sim.source_vector(t0).reshape(sim.mesh.n_elem, dz.dim, dz.Ng, dz.Nphi)
        assert np.abs(np.delete(sv, e_s, axis=0)).max() == 0.0
        for a in range(dz.Ng):
            def integrand(tau, a=a):
                return dz.tb.values(tau)[0, a] * ricker(t0 + tau * sim.dt, w.f0, w.t_delay, w.a1)
            ref = sim.dt * quad(integrand, 0.0, 1.0, epsabs=1e-15, epsrel=1e-13)[0]
            for k in range(dz.dim):
                got = sv[e_s, k, a].sum()
                assert abs(got - w.shots_dir[0][k] * ref) <= 1e-11 * sim.dt * w.a1, (t0, a, k, got, ref)


@pytest.mark.parametrize("scheme,p,pg", [("stdg", 2, 2), ("cn", 1, 0)])
def test_time_scaling_identity(scheme, p, pg):
    # A mesh part advancing with step alpha dt is the same discrete scheme as the part with
    # density rho / alpha, Lame parameters alpha lambda, alpha mu and the Ricker wavelet at
    # frequency alpha f0, delay t_D / alpha, advanced with step dt (Eq. 5 in the time
    # tau = t / alpha; the basis of per-part time steps in a ragged batch): states equal to
    # rounding, energy scaled by 1 / alpha
    w = synth.c4_ragged(0, steps=3, scale=0.02)
    alpha, dt = 1.7, w.dt
    direc = [0.3, 1.0]

    def run(lam, mu, rho, step, f0, td):
        sim = Simulation(w.xyz, w.elem_vert, w.period, lam, mu, rho, p, pg, scheme, step)
        sim.set_source(w.shots_xs[0], direc, f0, td, w.a1)
        sim.step(3)
        return sim

    a = run(w.lam, w.mu, w.rho, alpha * dt, w.f0, w.t_delay)
    b = run(alpha * w.lam, alpha * w.mu, w.rho / alpha, dt, alpha * w.f0, w.t_delay / alpha)
    assert np.abs(a.v_tr).max() > 0
    assert np.abs(b.v_tr - a.v_tr).max() <= 1e-10 * np.abs(a.v_tr).max()
    assert np.abs(b.sig_tr - a.sig_tr).max() <= 1e-10 * np.abs(a.sig_tr).max()
    assert abs(b.energy() - a.energy() / alpha) <= 1e-10 * a.energy()
    # a different step without the rescaling is a different solution
    c = run(w.lam, w.mu, w.rho, dt, w.f0, w.t_delay)
    assert np.abs(c.v_tr - a.v_tr).max() > 1e-3 * np.abs(a.v_tr).max()
