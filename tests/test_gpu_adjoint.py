"""Discrete adjoint of the step (sim_adjoint_*): gradients of the heat-release
objective and of a seeded state functional with respect to the slot burner's
profile coefficients, against central differences of the forward map (the
CUDA step itself, and the FP64 oracle).

FD step: the derivative along a unit direction of the coefficients (order
one) is only ~1e-4 J, so a step of 1e-6 leaves the quotient with ~1e-5
relative rounding noise (J itself carries ~1e-16 relative rounding); at
h = 1e-3 the truncation error is ~1e-8 relative (J is smooth in c) and the
noise ~1e-8.  The tolerance is 1e-6 relative; Poisson solves run to rtol 1e-13."""

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

FD_H = 1e-3
TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_01727_gb300 import build
    build.build()


def _case(nx=32, ny=64, n_bumps=8, n_profile=64):
    prm, geo, f, A, c = W.slot_bumps(nx, ny, n_bumps=n_bumps, n_profile=n_profile, Da_ib=(2.0 / nx) ** 2)
    prm["poisson_rtol"] = 1e-13
    prm["poisson_max_iter"] = 400
    return prm, geo, f, A, c


def _direction(m, seed=7):
    e = np.random.Generator(np.random.PCG64(seed)).standard_normal(m)
    return e / np.linalg.norm(e)


def test_heat_release_gradient_matches_central_differences():
    from paper_2603_01727_gb300.adjoint import HeatReleaseProblem
    prm, geo, f, A, c = _case()
    pb = HeatReleaseProblem(prm, geo, f, A, nsteps=12, every=5)
    J0 = pb.value(c)
    gc, gp = pb.gradient()
    assert J0 > 0.0 and np.all(np.isfinite(gc))
    e = _direction(len(c))
    fd = (pb.value(c + FD_H * e, False) - pb.value(c - FD_H * e, False)) / (2.0 * FD_H)
    ad = float(gc @ e)
    assert abs(fd - ad) <= TOL * abs(ad), (fd, ad)
    # single coefficients, and the profile-sample gradient through the basis
    for m in (0, len(c) // 2):
        em = np.zeros(len(c))
        em[m] = 1.0
        fdm = (pb.value(c + FD_H * em, False) - pb.value(c - FD_H * em, False)) / (2.0 * FD_H)
        assert abs(fdm - gc[m]) <= TOL * np.max(np.abs(gc)), (m, fdm, gc[m])
    assert np.allclose(A.T @ gp, gc, rtol=0, atol=1e-14 * np.max(np.abs(gc)))
    pb.close()


def test_differential_diffusion_gradient_matches_central_differences():
    """Le_F = 0.97, Le_O = 1.11 (the paper's values): the regularised
    Le_eps(Z) and N_eps(Z) of Eq 3.35 make the stage stencil depend on Z
    through its coefficients; the adjoint takes the exact dual-number gather
    of the stencil there.  Gradient along a random direction and two single
    coefficients within 1e-6 of central differences of the CUDA forward map."""
    from paper_2603_01727_gb300.adjoint import HeatReleaseProblem
    prm, geo, f, A, c = _case()
    prm.update(Le_F=0.97, Le_O=1.11)
    pb = HeatReleaseProblem(prm, geo, f, A, nsteps=12, every=5)
    J0 = pb.value(c)
    gc, _ = pb.gradient()
    assert J0 > 0.0 and np.all(np.isfinite(gc))
    e = _direction(len(c), seed=11)
    fd = (pb.value(c + FD_H * e, False) - pb.value(c - FD_H * e, False)) / (2.0 * FD_H)
    ad = float(gc @ e)
    assert abs(fd - ad) <= TOL * abs(ad), (fd, ad)
    for m in (1, len(c) - 2):
        em = np.zeros(len(c))
        em[m] = 1.0
        fdm = (pb.value(c + FD_H * em, False) - pb.value(c - FD_H * em, False)) / (2.0 * FD_H)
        assert abs(fdm - gc[m]) <= TOL * np.max(np.abs(gc)), (m, fdm, gc[m])
    pb.close()


def test_buoyancy_gradient_matches_central_differences():
    """inv_Fr2 = 1 (Eq 3.8b): the vertical momentum residual depends on the
    stage's density (rho^n in the predictor, rho* in the corrector), whose
    adjoint joins the density lambdas of the state relation.  Gradient along a
    random direction and a single coefficient within 1e-6 of central
    differences of the CUDA forward map, with and without differential
    diffusion."""
    from paper_2603_01727_gb300.adjoint import HeatReleaseProblem
    for lewis in ((1.0, 1.0), (0.97, 1.11)):
        prm, geo, f, A, c = _case()
        prm.update(inv_Fr2=1.0, Le_F=lewis[0], Le_O=lewis[1])
        pb = HeatReleaseProblem(prm, geo, f, A, nsteps=12, every=5)
        J0 = pb.value(c)
        gc, _ = pb.gradient()
        assert J0 > 0.0 and np.all(np.isfinite(gc))
        e = _direction(len(c), seed=13)
        fd = (pb.value(c + FD_H * e, False) - pb.value(c - FD_H * e, False)) / (2.0 * FD_H)
        ad = float(gc @ e)
        assert abs(fd - ad) <= TOL * abs(ad), (lewis, fd, ad)
        em = np.zeros(len(c))
        em[len(c) // 3] = 1.0
        fdm = (pb.value(c + FD_H * em, False) - pb.value(c - FD_H * em, False)) / (2.0 * FD_H)
        assert abs(fdm - gc[len(c) // 3]) <= TOL * np.max(np.abs(gc)), (lewis, fdm, gc[len(c) // 3])
        pb.close()


def test_sutherland_and_isothermal_walls_gradient_matches_central_differences():
    """Sutherland's law (Eq 4.12) in the state relation's transpose and
    isothermal side walls (Dirichlet Z and H, no-slip; their ghosts mirror
    about fixed values) in the ghost fills' transposes: the slot burner with
    both, gradient along a random direction within 1e-6 of central
    differences of the CUDA forward map."""
    from paper_2603_01727_gb300.adjoint import HeatReleaseProblem
    prm, geo, f, A, c = _case()
    S, Q, H_inf, _ = W.paper_scalars(prm["Z_st"], prm["density_ratio"])
    prm.update(transport=1, sutherland_C=110.5 / 600.0, bc=[[W.WALL_T, W.WALL_T]] + prm["bc"][1:],
               wall_H=[[H_inf, H_inf], [0.0, 0.0], [0.0, 0.0]])
    pb = HeatReleaseProblem(prm, geo, f, A, nsteps=12, every=5)
    J0 = pb.value(c)
    gc, _ = pb.gradient()
    assert J0 > 0.0 and np.all(np.isfinite(gc))
    e = _direction(len(c), seed=17)
    fd = (pb.value(c + FD_H * e, False) - pb.value(c - FD_H * e, False)) / (2.0 * FD_H)
    ad = float(gc @ e)
    assert abs(fd - ad) <= TOL * abs(ad), (fd, ad)
    pb.close()


def test_checkpoint_spacing_does_not_change_the_gradient():
    from paper_2603_01727_gb300.adjoint import HeatReleaseProblem
    prm, geo, f, A, c = _case(24, 48, 6, 32)
    grads = []
    for every in (1, 4, 50):
        pb = HeatReleaseProblem(prm, geo, f, A, nsteps=9, every=every)
        pb.value(c)
        grads.append(pb.gradient()[0])
        pb.close()
    for g in grads[1:]:
        assert np.array_equal(g, grads[0])


def test_seeded_state_functional_gradient():
    """Objective weight 0 and a seed on Z at the final level: the gradient of
    <w, Z^N> (and the adjoint field accessors)."""
    from paper_2603_01727_gb300.lowmach import Simulation
    prm, geo, f, A, c = _case(24, 48, 6, 32)
    N = 6
    w = np.random.Generator(np.random.PCG64(3)).standard_normal((48, 24))

    def run(cc, states=None):
        g = dict(geo, profile=list(A @ cc))
        sim = Simulation(prm, g)
        sim.set_fields(f)
        sim.step(0)
        for _ in range(N):
            if states is not None:
                buf = np.empty(sim.state_size(), dtype=np.uint8)
                sim.state_save(buf)
                states.append(buf)
            sim.step(1)
        sim.sync()
        return sim, float(np.sum(w * sim.get("Z")))

    states = []
    sim, _ = run(c, states)
    sim.adjoint_begin()
    sim.adjoint_seed("Z", w)
    assert np.array_equal(sim.adjoint_get("Z"), w)
    gp = None
    for n in range(N - 1, -1, -1):
        sim.state_load(states[n])
        gp = sim.adjoint_step(0.0, n_profile=A.shape[0])
    gc = A.T @ gp
    lz = sim.adjoint_get("Z")
    assert np.all(np.isfinite(lz)) and np.any(lz != 0.0)
    sim.adjoint_end()
    sim.close()
    e = _direction(len(c), seed=11)
    fp = run(c + FD_H * e)
    fm = run(c - FD_H * e)
    fd = (fp[1] - fm[1]) / (2.0 * FD_H)
    fp[0].close()
    fm[0].close()
    ad = float(gc @ e)
    assert abs(fd - ad) <= TOL * abs(ad), (fd, ad)


def test_adjoint_gradient_matches_oracle_differences():
    """The GPU adjoint's directional derivative against central differences of
    the FP64 oracle's objective (its own step and exact transform Poisson)."""
    from oracle import objective as O
    from oracle import step as S
    from paper_2603_01727_gb300.adjoint import HeatReleaseProblem
    prm, geo, f, A, c = _case(24, 48, 6, 32)
    N = 6
    pb = HeatReleaseProblem(prm, geo, f, A, nsteps=N, every=3)
    Jg = pb.value(c)
    gc, _ = pb.gradient()
    pb.close()
    e = _direction(len(c), seed=5)

    def J_oracle(cc):
        p = S.Problem(prm, dict(geo, profile=list(A @ cc)))
        st = S.initial_state(p, f["v"], f["Z"], f["H"])
        return O.objective(p, st, N, S.advance)

    J0 = J_oracle(c)
    assert abs(J0 - Jg) <= 1e-9 * abs(J0)
    fd = (J_oracle(c + FD_H * e) - J_oracle(c - FD_H * e)) / (2.0 * FD_H)
    ad = float(gc @ e)
    assert abs(fd - ad) <= TOL * abs(ad), (fd, ad)


def test_adjoint_rejects_unsupported_configurations():
    from paper_2603_01727_gb300.lowmach import Simulation, SimError, SIM_EINVAL
    prm, geo, f, A, c = _case(24, 48, 6, 32)
    prm = dict(prm, precision=W.MIXED)
    sim = Simulation(prm, geo)
    sim.set_fields(f)
    sim.step(1)
    with pytest.raises(SimError) as e:
        sim.adjoint_begin()
    assert e.value.status == SIM_EINVAL
    sim.close()


@pytest.mark.parametrize("lewis", [1.0, 1.1])
def test_reverse_stencil_matches_dual_number_gather(lewis, monkeypatch):
    """The hand-written reverse sweep of the stage stencil against the exact
    dual-number gather (LOWMACH_ADJ_DUAL=1): every adjoint field after two
    reverse steps seeded by the objective and a random Z seed.  Le_F = Le_O =
    1.1 exercises the N_O dZ term of the H equation."""
    from paper_2603_01727_gb300.lowmach import Simulation
    prm, geo, f, A, c = _case(24, 48, 6, 32)
    prm = dict(prm, Le_F=lewis, Le_O=lewis)
    w = np.random.Generator(np.random.PCG64(9)).standard_normal((48, 24))
    names = ["U", "V", "Z", "H", "T", "RHO", "KAPPA", "FX", "FY", "SM"]
    out = {}
    for dual in ("0", "1"):
        monkeypatch.setenv("LOWMACH_ADJ_DUAL", dual)
        sim = Simulation(prm, geo)
        sim.set_fields(f)
        sim.step(3)
        states = []
        for _ in range(2):
            buf = np.empty(sim.state_size(), dtype=np.uint8)
            sim.state_save(buf)
            states.append(buf)
            sim.step(1)
        sim.adjoint_begin()
        sim.adjoint_seed("Z", w)
        gp = None
        for n in (1, 0):
            sim.state_load(states[n])
            gp = sim.adjoint_step(prm["dt"], n_profile=A.shape[0])
        out[dual] = {k: sim.adjoint_get(k) for k in names}
        out[dual]["profile"] = gp
        sim.adjoint_end()
        sim.close()
    for k in names + ["profile"]:
        a, b = out["0"][k], out["1"][k]
        scale = np.max(np.abs(b))
        assert scale > 0.0, k
        assert np.max(np.abs(a - b)) <= 1e-12 * scale, (k, np.max(np.abs(a - b)) / scale)


def test_autograd_function_matches_problem_gradient():
    """The torch.autograd.Function wrapper: J from forward() and dJ/dc from
    torch.autograd are bit for bit those of HeatReleaseProblem.value /
    .gradient, and the chain rule through the Function holds."""
    import torch
    from paper_2603_01727_gb300.adjoint import HeatReleaseProblem, heat_release_function
    prm, geo, f, A, c = _case(24, 48, 6, 32)
    pb = HeatReleaseProblem(prm, geo, f, A, nsteps=8, every=3)
    HR = heat_release_function()
    ct = torch.tensor(c, dtype=torch.float64, requires_grad=True)
    J = HR.apply(ct, pb)
    (gt,) = torch.autograd.grad(J, ct)
    J_ref = pb.value(c)
    g_ref, _ = pb.gradient()
    assert float(J.detach()) == J_ref
    assert np.array_equal(gt.numpy(), g_ref)
    ct2 = torch.tensor(c, dtype=torch.float64, requires_grad=True)
    loss = 3.0 * HR.apply(ct2, pb) ** 2
    loss.backward()
    assert np.allclose(ct2.grad.numpy(), 6.0 * J_ref * g_ref, rtol=1e-15, atol=0.0)
    pb.close()


def test_c4_configuration_gradient():
    """The adjoint configuration itself: the 128x256 slot burner whose flux
    profile is 64 Gaussian bumps, J over 200 steps, checkpoints every 20.  The
    adjoint gradient against central differences of the CUDA forward map along
    a random direction and for three single coefficients; J against the FP64
    oracle's J at the same coefficients."""
    from oracle import objective as O
    from oracle import step as S
    from paper_2603_01727_gb300.adjoint import HeatReleaseProblem
    prm, geo, f, A, c = W.slot_bumps()
    prm["poisson_rtol"] = 1e-13
    prm["poisson_max_iter"] = 400
    N = 200
    pb = HeatReleaseProblem(prm, geo, f, A, nsteps=N, every=20)
    J = pb.value(c)
    gc, _ = pb.gradient()
    assert J > 0.0 and np.all(np.isfinite(gc))

    def fd(e, h=1e-2):
        # Over 200 steps a unit direction moves J by only ~5e-6 of itself, so
        # at h = 1e-3 the quotient's rounding noise is ~1e-6 relative.  Central
        # differences at h and 2h, Richardson-combined (error O(h^4)), keep
        # both the noise and the truncation error near 1e-8.
        d = lambda hh: (pb.value(c + hh * e, False) - pb.value(c - hh * e, False)) / (2.0 * hh)
        return (4.0 * d(h) - d(2.0 * h)) / 3.0

    e = _direction(len(c), seed=13)
    fdv = fd(e)
    ad = float(gc @ e)
    print("c4 direction: adjoint", ad, "fd", fdv, "rel", abs(fdv - ad) / abs(ad))
    assert abs(fdv - ad) <= TOL * abs(ad), (fdv, ad)
    for m in (0, 31, 63):
        em = np.zeros(len(c))
        em[m] = 1.0
        fdm = fd(em)
        print("c4 coefficient", m, "adjoint", gc[m], "fd", fdm, "rel", abs(fdm - gc[m]) / np.max(np.abs(gc)))
        assert abs(fdm - gc[m]) <= TOL * np.max(np.abs(gc)), (m, fdm, gc[m])
    pb.close()
    p = S.Problem(prm, dict(geo, profile=list(A @ c)))
    st = S.initial_state(p, f["v"], f["Z"], f["H"])
    J_oracle = O.objective(p, st, N, S.advance)
    print("c4 J", J, "oracle", J_oracle)
    assert abs(J_oracle - J) <= 1e-9 * abs(J_oracle)
