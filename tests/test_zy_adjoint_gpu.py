"""GPU misfit gradient (stdg_misfit_grad) against the oracle's discrete adjoint and
against central finite differences of the GPU's own misfit."""
import numpy as np
import pytest

import synth
from helpers import gpu_solver, need_gpu

pytestmark = pytest.mark.gpu


def _case(p=1, ny=5, steps=12, n_shots=2, n_rec=6):
    w = synth.c5_adjoint(ny=ny, p=p, steps=steps, n_shots=n_shots, n_rec=n_rec)
    wt = synth.c5_adjoint(ny=ny, p=p, steps=steps, n_shots=n_shots, n_rec=n_rec, true_model=True)
    return w, wt


def _oracle(w, wt):
    from oracle import adjoint as adj
    geom = (w.xyz, w.elem_vert, w.period, w.p, w.p_gamma, w.dt)
    geom_t = (wt.xyz, wt.elem_vert, wt.period, wt.p, wt.p_gamma, wt.dt)
    src = [(w.shots_xs[k], w.shots_dir[k]) for k in range(w.n_shots)]
    data = np.array([adj.forward(adj.make_sim(geom_t, wt.lam, wt.mu, wt.rho), w.n_steps, s, w.f0, w.t_delay, w.a1,
                                 w.receivers)[0] for s in src])
    return data, adj.misfit_gradient(geom, w.lam, w.mu, w.rho, w.n_steps, src, w.f0, w.t_delay, w.a1,
                                     w.receivers, data)


@pytest.mark.parametrize("p,precision,pre,ckpt", [(1, "fp64", 2, 5), (2, "fp64", 1, 20), (2, "mixed", 2, 4)])
def test_misfit_gradient_matches_oracle(p, precision, pre, ckpt):
    need_gpu()
    w, wt = _case(p=p)
    data, (L, gl, gm, gr) = _oracle(w, wt)
    rel_tol = 1e-13 if precision == "fp64" else 1e-12
    s = gpu_solver(w, precision=precision, rel_tol=rel_tol, max_iters=20000, preconditioner=pre)
    Lg, glg, gmg, grg, st = s.misfit_grad(w.dt, w.n_steps, data, checkpoint_every=ckpt)
    # The residual rec - d of a small model perturbation cancels: a relative error e of the
    # records becomes e * amp in the residual, amp = |d| / |rec - d|.  The bar is the solve
    # tolerance's reach times that amplification (FP64 1e-13 solves, mixed 1e-12).
    amp = np.linalg.norm(data) / np.sqrt(2.0 * L)
    tol = (1e-11 if precision == "fp64" else 1e-10) * amp + 1e-10
    errs = [np.abs(a - b).max() / np.abs(b).max() for a, b in ((glg, gl), (gmg, gm), (grg, gr))]
    print(p, precision, pre, "amp %.3g tol %.3g loss err %.3g grad errs" % (amp, tol, abs(Lg - L) / L), errs)
    assert abs(Lg - L) <= tol * L
    assert max(errs) <= tol
    # the context ends at the final time with the forward run's final states
    f = gpu_solver(w, precision=precision, rel_tol=rel_tol, max_iters=20000, preconditioner=pre)
    f.step(w.dt, w.n_steps)
    for k in range(w.n_shots):
        v1, s1 = s.get_state(k)
        v2, s2 = f.get_state(k)
        assert np.abs(v1 - v2).max() <= 1e-10 * np.abs(v2).max()


def test_misfit_gradient_matches_gpu_finite_differences():
    # the GPU's own misfit, FP64 solves to 1e-14, Richardson-extrapolated central differences
    need_gpu()
    w, wt = _case(p=2, steps=10)
    data, _ = _oracle(w, wt)
    s = gpu_solver(w, precision="fp64", rel_tol=1e-14, max_iters=20000, preconditioner=2)
    _, gl, gm, gr, _ = s.misfit_grad(w.dt, w.n_steps, data, checkpoint_every=3)
    rng = np.random.default_rng(4)
    for name, g in (("lam", gl), ("mu", gm), ("rho", gr)):
        big = np.where(np.abs(g) >= 1e-2 * np.abs(g).max())[0]
        for e in rng.choice(big, 2, replace=False):
            fds = []
            for hr in (1e-4, 0.5e-4):
                Ls = []
                for sgn in (1.0, -1.0):
                    q = {"lam": w.lam.copy(), "mu": w.mu.copy(), "rho": w.rho.copy()}
                    q[name][e] *= 1.0 + sgn * hr
                    f = gpu_solver(w, precision="fp64", rel_tol=1e-14, max_iters=20000, preconditioner=2)
                    f.set_material(q["lam"], q["mu"], q["rho"])
                    f.set_sources(w.shots_xs, w.shots_dir, w.f0, w.t_delay, w.a1)
                    Ls.append(f.misfit_grad(w.dt, w.n_steps, data, grad=False)[0])
                fds.append((Ls[0] - Ls[1]) / (2 * hr * {"lam": w.lam, "mu": w.mu, "rho": w.rho}[name][e]))
            fd = (4.0 * fds[1] - fds[0]) / 3.0
            assert abs(fd - g[e]) <= 1e-6 * abs(g[e]) + 1e-9 * np.abs(g).max(), (name, e, fd, g[e])


def test_autograd_function_returns_the_adjoint_gradient():
    import torch
    from paper_1802_04516_gb300.binding import misfit
    need_gpu()
    w, wt = _case(p=1, steps=8)
    data, (L, gl, gm, gr) = _oracle(w, wt)
    s = gpu_solver(w, precision="fp64", rel_tol=1e-13, max_iters=20000, preconditioner=2)
    lam = torch.tensor(w.lam, requires_grad=True)
    mu = torch.tensor(w.mu, requires_grad=True)
    rho = torch.tensor(w.rho, requires_grad=True)
    loss = misfit(s, lam, mu, rho, w.dt, w.n_steps, data,
                  reset=lambda: s.set_sources(w.shots_xs, w.shots_dir, w.f0, w.t_delay, w.a1))
    (3.0 * loss).backward()
    amp = np.linalg.norm(data) / np.sqrt(2.0 * L)
    tol = 1e-11 * amp + 1e-10
    assert abs(loss.item() - L) <= tol * L
    for t, g in ((lam, gl), (mu, gm), (rho, gr)):
        assert np.abs(t.grad.numpy() - 3.0 * g).max() <= tol * np.abs(3.0 * g).max()


def test_source_gradient_matches_oracle():
    # dL/d(amplitude, force direction, position) of every shot's point source (Sec. 6.3),
    # against the oracle's discrete adjoint; the bar as for the material gradients
    need_gpu()
    from oracle import adjoint as adj
    w, wt = _case(p=2)
    data, _ = _oracle(w, wt)
    geom = (w.xyz, w.elem_vert, w.period, w.p, w.p_gamma, w.dt)
    src = [(w.shots_xs[k], w.shots_dir[k]) for k in range(w.n_shots)]
    L, _, _, _, gs = adj.misfit_gradient(geom, w.lam, w.mu, w.rho, w.n_steps, src, w.f0, w.t_delay, w.a1,
                                         w.receivers, data, source_grad=True)
    for precision, rel_tol in (("fp64", 1e-13), ("mixed", 1e-12)):
        s = gpu_solver(w, precision=precision, rel_tol=rel_tol, max_iters=20000, preconditioner=2)
        Lg, _, _, _, gsg, _ = s.misfit_grad(w.dt, w.n_steps, data, checkpoint_every=5, source_grad=True)
        amp = np.linalg.norm(data) / np.sqrt(2.0 * L)
        tol = (1e-11 if precision == "fp64" else 1e-10) * amp + 1e-10
        err = np.abs(gsg - gs).max() / np.abs(gs).max()
        print(precision, "source gradient error %.3g (bar %.3g)" % (err, tol))
        assert gsg.shape == gs.shape and err <= tol


def test_source_gradient_matches_gpu_finite_differences():
    # the GPU's own misfit with FP64 solves to 1e-14: the misfit is quadratic in the force
    # direction (exact central differences) and smooth in the position inside the source's
    # element (Richardson-extrapolated differences); a1 dL/da1 = d . dL/dd
    need_gpu()
    w, wt = _case(p=2, steps=10)
    data, _ = _oracle(w, wt)
    s = gpu_solver(w, precision="fp64", rel_tol=1e-14, max_iters=20000, preconditioner=2)
    _, _, _, _, gs, _ = s.misfit_grad(w.dt, w.n_steps, data, checkpoint_every=4, source_grad=True)
    d = w.dim

    def L(xs, dr):
        f = gpu_solver(w, precision="fp64", rel_tol=1e-14, max_iters=20000, preconditioner=2)
        f.set_sources(xs, dr, w.f0, w.t_delay, w.a1)
        return f.misfit_grad(w.dt, w.n_steps, data, grad=False)[0]

    for k in range(w.n_shots):
        g = gs[k]
        assert abs(w.a1 * g[0] - w.shots_dir[k] @ g[1:1 + d]) <= 1e-9 * np.abs(w.a1 * g[0])
        for l in range(d):
            dp, dm = w.shots_dir.copy(), w.shots_dir.copy()
            dp[k, l] += 1e-3
            dm[k, l] -= 1e-3
            fd = (L(w.shots_xs, dp) - L(w.shots_xs, dm)) / 2e-3
            assert abs(fd - g[1 + l]) <= 1e-6 * np.abs(g[1:1 + d]).max(), ("dir", k, l, fd, g[1 + l])
            fds = []
            for hx in (2e-5, 1e-5):
                xp, xm = w.shots_xs.copy(), w.shots_xs.copy()
                xp[k, l] += hx
                xm[k, l] -= hx
                fds.append((L(xp, w.shots_dir) - L(xm, w.shots_dir)) / (2 * hx))
            fd = (4.0 * fds[1] - fds[0]) / 3.0
            assert abs(fd - g[1 + d + l]) <= 1e-5 * np.abs(g[1 + d:]).max(), ("x_s", k, l, fd, g[1 + d + l])


def test_autograd_function_differentiates_the_sources():
    import torch
    from paper_1802_04516_gb300.binding import misfit
    need_gpu()
    w, wt = _case(p=1, steps=8)
    data, _ = _oracle(w, wt)
    s = gpu_solver(w, precision="fp64", rel_tol=1e-13, max_iters=20000, preconditioner=2)
    force = w.a1 * w.shots_dir
    lam, mu, rho = (torch.tensor(a, requires_grad=True) for a in (w.lam, w.mu, w.rho))
    xs = torch.tensor(w.shots_xs, requires_grad=True)
    fo = torch.tensor(force, requires_grad=True)
    loss = misfit(s, lam, mu, rho, w.dt, w.n_steps, data,
                  sources=dict(xs=xs, force=fo, f0=w.f0, t_delay=w.t_delay, n_shots=w.n_shots))
    (2.0 * loss).backward()
    ref = gpu_solver(w, precision="fp64", rel_tol=1e-13, max_iters=20000, preconditioner=2)
    Lr, gl, _, _, gs, _ = ref.misfit_grad(w.dt, w.n_steps, data, source_grad=True)
    d = w.dim
    assert abs(loss.item() - Lr) <= 1e-10 * Lr
    assert np.abs(xs.grad.numpy() - 2.0 * gs[:, 1 + d:]).max() <= 1e-9 * np.abs(gs[:, 1 + d:]).max()
    assert np.abs(fo.grad.numpy() - 2.0 * gs[:, 1:1 + d] / w.a1).max() <= 1e-9 * np.abs(gs[:, 1:1 + d]).max()
    assert np.abs(lam.grad.numpy() - 2.0 * gl).max() <= 1e-9 * np.abs(gl).max()
