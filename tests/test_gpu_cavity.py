"""Differentially heated cavity (Sec. 4.3): isothermal walls (Eq 4.16a-b) and
Sutherland transport (Eq 4.12) on the GPU, against the oracle and against the
paper's converged hydrodynamic pressure and Nusselt numbers at Ra = 1e2
(Tables 3 and 5).
"""

import numpy as np
import pytest

import workloads as W
from oracle import step as S
from oracle.operators import V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_01727_gb300 import build
    build.build()


def rel(a, b):
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / (scale if scale > 0 else 1.0)


def _oracle(prm, geo, f, steps):
    pb = S.Problem(prm, geo)
    st = S.initial_state(pb, f["v"], f["Z"], f["H"])
    for _ in range(steps):
        st = S.advance(pb, st)
    g = pb.g
    out = {"UVW"[d]: V(st.v[d], g) for d in range(g.dim)}
    out.update(Z=V(st.Z, g), H=V(st.H, g), T=V(st.T, g), RHO=V(st.rho, g), P=V(st.P, g),
               KAPPA=V(st.kappa, g))
    for d in range(g.dim):
        out["F" + "XYZ"[d]] = V(st.F[d], g, face=d)
    return out, st.p0_hist[0]


def _gpu(prm, geo, f, steps):
    from paper_2603_01727_gb300.lowmach import Simulation
    sim = Simulation(prm, geo)
    sim.set_fields(f)
    sim.step(steps)
    sim.sync()
    return sim


@pytest.mark.parametrize("n,steps,gravity", [(32, 150, True), (40, 60, True), (24, 100, False)])
def test_heated_cavity_matches_oracle(n, steps, gravity):
    """Every field and p0 after `steps` FP64 steps within 1e-9 of the oracle."""
    from paper_2603_01727_gb300.lowmach import SIM_Q_P0
    prm, geo, f = W.heated_cavity(n, gravity=gravity, ny=None if gravity else 8)
    prm["poisson_rtol"] = 1e-13
    ref, p0 = _oracle(prm, geo, f, steps)
    sim = _gpu(prm, geo, f, steps)
    worst = {k: rel(sim.get(k), v) for k, v in ref.items()}
    bad = {k: e for k, e in worst.items() if not e <= 1e-9}
    assert not bad, (bad, worst)
    assert sim.query(SIM_Q_P0) == pytest.approx(p0, rel=1e-12)
    sim.close()


def test_heated_cavity_mixed_precision_against_oracle():
    """The mixed path on the cavity: within the bound the other mixed-precision
    checks use (the stage kernels' float-float error, amplified by 150 steps)."""
    prm, geo, f = W.heated_cavity(32)
    prm.update(poisson_rtol=1e-12, precision=W.MIXED)
    ref, _ = _oracle(dict(prm, precision=W.FP64), geo, f, 150)
    sim = _gpu(prm, geo, f, 150)
    worst = {k: rel(sim.get(k), v) for k, v in ref.items()}
    print("mixed", {k: f"{v:.1e}" for k, v in worst.items()})
    bad = {k: e for k, e in worst.items() if not e <= 1e-6}
    assert not bad, (bad, worst)
    sim.close()


def _nusselt_middle(T, KAPPA, FX, prm, eps):
    """Average Nusselt number on the vertical mid-line x_1 = 1/2 (Eqs 4.14,
    4.15): (Pe rho v_1 T - kappa dT/dx_1) / (2 eps) on the faces there (the
    mass flux F_1 is rho v_1 on the face), averaged over x_2."""
    n = prm["n"][0]
    m = n // 2
    Pe = prm["Re"] * prm["Pr"]
    Tf = 0.5 * (T[:, m - 1] + T[:, m])
    kf = 0.5 * (KAPPA[:, m - 1] + KAPPA[:, m])
    return float(np.mean(Pe * FX[:, m] * Tf - kf * (T[:, m] - T[:, m - 1]) * n) / (2.0 * eps))


def test_heated_cavity_ra1e2_steady_state_matches_table5():
    """Ra = 1e2, eps = 0.6 run to steady state on 48^2 and 72^2 uniform grids
    (refinement ratio 1.5, as in the grid study of Table 3), then Richardson
    extrapolated at second order: p0 within 3e-5 of both the paper's value
    (0.95738) and its reference value (0.95736) of Table 5, and the mid-line
    Nusselt number within 2e-4 of theirs (0.9787)."""
    from paper_2603_01727_gb300.lowmach import SIM_Q_P0
    eps, t_end = 0.6, 8.0
    p0, nu = [], []
    for n in (48, 72):
        prm, geo, f = W.heated_cavity(n, Ra=1e2, eps=eps, cfl=0.7)
        sim = _gpu(prm, geo, f, int(np.ceil(t_end / prm["dt"])))
        p0.append(sim.query(SIM_Q_P0))
        nu.append(_nusselt_middle(sim.get("T"), sim.get("KAPPA"), sim.get("FX"), prm, eps))
        sim.close()
    r2 = 1.5 ** 2
    p_inf = p0[1] + (p0[1] - p0[0]) / (r2 - 1.0)
    nu_inf = nu[1] + (nu[1] - nu[0]) / (r2 - 1.0)
    print("p0", p0, "extrapolated", p_inf, "Nu_M", nu, "extrapolated", nu_inf)
    assert p0[0] > p0[1] > p_inf                     # monotone approach from above, as in Table 3
    assert abs(p_inf - 0.95738) < 3e-5 and abs(p_inf - 0.95736) < 3e-5
    assert abs(nu_inf - 0.9787) < 2e-4
