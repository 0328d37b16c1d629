"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

Tolerances: relative L-infinity by field maximum, max|gpu - oracle| / max|oracle|.
FP64 everywhere; the only differences are rounding order (reductions, fused
multiply-adds) and the pressure solve, which is iterative on the GPU
(poisson_rtol) and exact on the oracle.  With poisson_rtol = 1e-13 every field
agrees within 1e-9 after 100 steps (the parity target); at the timing tolerance
1e-10 the bound is derived in each test from the residual bound.
"""

import os

import numpy as np
import pytest

import workloads as W
from oracle import step as S
from oracle import poisson as OP
from oracle.operators import V

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_01727_gb300 import build
    build.build()


def _torch():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def rel(a, b):
    scale = float(np.max(np.abs(b)))
    return float(np.max(np.abs(a - b))) / (scale if scale > 0 else 1.0)


def oracle_run(prm, geo, f, nsteps):
    pb = S.Problem(prm, geo)
    st = S.initial_state(pb, f["v"], f["Z"], f["H"])
    for _ in range(nsteps):
        st = S.advance(pb, st)
    return pb, st


def oracle_fields(pb, st):
    g = pb.g
    out = {"UVW"[d]: V(st.v[d], g) for d in range(g.dim)}
    out.update(Z=V(st.Z, g), H=V(st.H, g), T=V(st.T, g), RHO=V(st.rho, g), P=V(st.P, g),
               KAPPA=V(st.kappa, g))
    for d in range(g.dim):
        out["F" + "XYZ"[d]] = V(st.F[d], g, face=d)
    return out


def gpu_run(prm, geo, f, nsteps):
    from paper_2603_01727_gb300.lowmach import Simulation
    sim = Simulation(prm, geo)
    sim.set_fields(f)
    sim.step(nsteps)
    sim.sync()
    return sim


def compare(sim, ref, tol, names=None):
    worst = {}
    for k, v in ref.items():
        if names is not None and k not in names:
            continue
        worst[k] = rel(sim.get(k), v)
    bad = {k: e for k, e in worst.items() if not e <= tol}
    assert not bad, (bad, worst)
    return worst


# ---------------------------------------------------------------------------
# Poisson solve (the dominant kernel) against the exact transform solve
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,periodic", [
    ((64, 64), (1, 1)), ((256, 512), (1, 0)), ((96, 40), (0, 0)), ((50, 50), (1, 1)),
    ((12, 20), (0, 1)), ((24, 16, 20), (0, 0, 0)), ((32, 32, 32), (1, 0, 1)), ((8, 8), (0, 0))])
def test_poisson_solve_matches_transform_solve(n, periodic):
    torch = _torch()
    from paper_2603_01727_gb300.lowmach import poisson_solve
    from oracle.operators import Grid
    rng = np.random.Generator(np.random.PCG64(11))
    L = [1.0 + 0.25 * d for d in range(len(n))]
    g = Grid(n, L)
    b = rng.normal(size=tuple(reversed(n)))
    ref = OP.solve(b, g, periodic)
    bt = torch.tensor(b, device="cuda", dtype=torch.float64)
    Pt = torch.zeros_like(bt)
    it, rr = poisson_solve(bt, Pt, g.h, periodic, rtol=1e-13, max_iter=300)
    assert rr <= 1e-13
    P = Pt.cpu().numpy()
    assert abs(P.mean()) < 1e-12 * np.abs(ref).max()
    assert rel(P, ref) < 1e-9, (rel(P, ref), it)
    # warm start from the answer converges immediately
    it2, _ = poisson_solve(bt, Pt, g.h, periodic, rtol=1e-10, max_iter=300)
    assert it2 <= 1


def test_poisson_solve_into_misaligned_views():
    """The solution array of the caller need not be 16-byte aligned: a view at
    an 8-byte offset takes the scalar update path and gives the same answer."""
    torch = _torch()
    from paper_2603_01727_gb300.lowmach import poisson_solve
    n, periodic = (64, 32), (1, 0)
    rng = np.random.Generator(np.random.PCG64(21))
    b = rng.normal(size=(n[1], n[0]))
    h = (1.0 / n[0], 0.5 / n[1])
    bt = torch.tensor(b, device="cuda", dtype=torch.float64)
    P0 = torch.zeros_like(bt)
    poisson_solve(bt, P0, h, periodic, rtol=1e-12, max_iter=300)
    big = torch.zeros(n[0] * n[1] + 1, dtype=torch.float64, device="cuda")
    P1 = big[1:].view(n[1], n[0])
    assert P1.data_ptr() % 16 == 8
    poisson_solve(bt, P1, h, periodic, rtol=1e-12, max_iter=300)
    assert rel(P1.cpu().numpy(), P0.cpu().numpy()) < 1e-11


def test_poisson_zero_rhs_gives_zero():
    torch = _torch()
    from paper_2603_01727_gb300.lowmach import poisson_solve
    b = torch.zeros((16, 16), dtype=torch.float64, device="cuda")
    P = torch.randn((16, 16), dtype=torch.float64, device="cuda")
    poisson_solve(b, P, (1 / 16, 1 / 16), (1, 1), rtol=1e-10)
    assert float(P.abs().max()) == 0.0


# ---------------------------------------------------------------------------
# Whole steps
# ---------------------------------------------------------------------------
def test_taylor_green_steps_match_oracle():
    prm, geo, f = W.taylor_green(50, 4e-3)
    pb, st = oracle_run(prm, geo, f, 20)
    sim = gpu_run(prm, geo, f, 20)
    compare(sim, oracle_fields(pb, st), 1e-11, names=["U", "V", "P", "FX", "FY"])


def test_periodic_blobs_100_steps_within_1e9():
    """Enclosed 64x64 box, 100 steps: every field within 1e-9 (parity target)."""
    prm, geo, f = W.periodic_blobs(64)
    prm["poisson_rtol"] = 1e-13
    pb, st = oracle_run(prm, geo, f, 100)
    sim = gpu_run(prm, geo, f, 100)
    worst = compare(sim, oracle_fields(pb, st), 1e-9)
    assert sim.query(2) == pytest.approx(st.p0_hist[0], rel=1e-12)   # p0
    print(worst)


@pytest.mark.parametrize("nx,ny,steps", [(32, 64, 30), (64, 128, 20), (48, 96, 10)])
def test_slot_burner_matches_oracle(nx, ny, steps):
    prm, geo, f = W.slot_burner(nx, ny)
    prm["poisson_rtol"] = 1e-13
    pb, st = oracle_run(prm, geo, f, steps)
    sim = gpu_run(prm, geo, f, steps)
    compare(sim, oracle_fields(pb, st), 1e-9)
    # immersed-body data: the mask is integer work, bit-exact
    chi = sim.get("CHI")
    assert np.array_equal(chi, V(pb.ibm["chi"], pb.g))
    assert rel(sim.get("SM"), pb.ibm["Sm"]) < 1e-14


# Method variants: differential diffusion with the paper's Lewis numbers
# (Le_F = 0.97, Le_O = 1.11; regularised Le_eps and N_eps of Eq 3.35) and the
# buoyancy term of Eq 3.8b, on the slot burner and the enclosed box.
@pytest.mark.parametrize("case", ["lewis_slot", "lewis_box", "buoyant_slot", "buoyant_lewis_box"])
def test_method_variants_match_oracle(case):
    if case.endswith("slot"):
        prm, geo, f = W.slot_burner(32, 64)
        steps = 20
    else:
        prm, geo, f = W.periodic_blobs(48)
        steps = 30
    if "lewis" in case:
        prm.update(Le_F=0.97, Le_O=1.11)
    if "buoyant" in case:
        prm["inv_Fr2"] = 1.0
    prm["poisson_rtol"] = 1e-13
    pb, st = oracle_run(prm, geo, f, steps)
    sim = gpu_run(prm, geo, f, steps)
    worst = compare(sim, oracle_fields(pb, st), 1e-9)
    print(case, {k: f"{v:.1e}" for k, v in worst.items()})


@pytest.mark.parametrize("case", ["lewis_slot", "buoyant_lewis_box"])
def test_method_variants_mixed_precision_error(case):
    if case.endswith("slot"):
        prm, geo, f = W.slot_burner(32, 64)
        steps = 20
        prm.update(Le_F=0.97, Le_O=1.11)
    else:
        prm, geo, f = W.periodic_blobs(48)
        steps = 30
        prm.update(Le_F=0.97, Le_O=1.11, inv_Fr2=1.0)
    prm["poisson_rtol"] = 1e-12
    prm["precision"] = W.MIXED
    pb, st = oracle_run(prm, geo, f, steps)
    sim = gpu_run(prm, geo, f, steps)
    worst = compare(sim, oracle_fields(pb, st), MIXED_TOL)
    print(case, {k: f"{v:.1e}" for k, v in worst.items()})


@pytest.mark.parametrize("case,precision", [("blobs", W.FP64), ("filling", W.FP64), ("filling", W.MIXED),
                                            ("filling3d", W.FP64)])
def test_semi_enclosed_p0_ode_matches_oracle(case, precision):
    """closed_system = 2: p0 advanced by the ODE of Eq 2.38 in the stages.  A
    burning closed box and a chamber filled through its bottom side; FP64
    within 1e-9 of the oracle (fields and p0), mixed within the mixed bound."""
    from paper_2603_01727_gb300.lowmach import SIM_Q_P0
    if case == "blobs":
        prm, geo, f = W.periodic_blobs(32)
        prm["closed_system"] = 2
        steps = 40
    elif case == "filling":
        prm, geo, f = W.filling_chamber(32)
        steps = 40
    else:
        prm, geo, f = W.filling_chamber(16, dim=3)
        steps = 12
    prm.update(poisson_rtol=1e-13 if precision == W.FP64 else 1e-12, precision=precision)
    pb, st = oracle_run(dict(prm, precision=W.FP64), geo, f, steps)
    assert st.p0_hist[0] > 1.05
    sim = gpu_run(prm, geo, f, steps)
    tol = 1e-9 if precision == W.FP64 else MIXED_TOL
    worst = compare(sim, oracle_fields(pb, st), tol)
    assert sim.query(SIM_Q_P0) == pytest.approx(st.p0_hist[0], rel=tol)
    print(case, precision, {k: f"{v:.1e}" for k, v in worst.items()})
    sim.close()


def test_semi_enclosed_restart_carries_the_ode_history():
    """The AB2 predictor of Eq 2.38 needs G of the previous level: a run saved
    and reloaded mid-way steps to the same bits as the uninterrupted run."""
    prm, geo, f = W.filling_chamber(32)
    sim = gpu_run(prm, geo, f, 6)
    blob = np.zeros(sim.state_size(), dtype=np.uint8)
    sim.state_save(blob)
    sim.step(5)
    sim.sync()
    ref = {k: sim.get(k) for k in ("U", "V", "Z", "H", "P", "RHO")}
    sim.state_load(blob)
    sim.step(5)
    sim.sync()
    for k, v in ref.items():
        assert np.array_equal(sim.get(k), v), k
    sim.close()


def test_semi_enclosed_rejects_outflow_and_bodies():
    from paper_2603_01727_gb300.lowmach import Simulation, SimError
    prm, geo, f = W.filling_chamber(16)
    bad = dict(prm, bc=[[W.PERIODIC, W.PERIODIC], [W.INFLOW, W.OUTFLOW], [W.PERIODIC, W.PERIODIC]])
    with pytest.raises(SimError):
        Simulation(bad, None)
    _, sgeo, _ = W.slot_burner(32, 64)
    with pytest.raises(SimError):
        Simulation(prm, sgeo)


def test_sphere_burner_3d_matches_oracle():
    prm, geo, f = W.sphere_burner(24)
    prm["poisson_rtol"] = 1e-13
    pb, st = oracle_run(prm, geo, f, 6)
    sim = gpu_run(prm, geo, f, 6)
    compare(sim, oracle_fields(pb, st), 1e-9)
    assert np.array_equal(sim.get("CHI"), V(pb.ibm["chi"], pb.g))


def test_slot_burner_full_size_timing_tolerance():
    """256x512 in the bench's configuration (poisson_rtol = 1e-10, graphs on),
    4 steps.  The pressure error of an iterative solve is bounded by
    cond(A) * rtol relative; the velocity and flux follow through the gradient,
    the scalars through one more stage, hence the looser bound for P, v, F."""
    prm, geo, f = W.slot_burner()
    pb, st = oracle_run(prm, geo, f, 4)
    sim = gpu_run(prm, geo, f, 4)
    ref = oracle_fields(pb, st)
    compare(sim, ref, 1e-9, names=["Z", "H", "T", "RHO", "KAPPA"])
    compare(sim, ref, 1e-6, names=["U", "V", "P", "FX", "FY"])
    assert sim.query(7) <= 1e-10 and sim.query(6) <= 1e-10


# ---------------------------------------------------------------------------
# Mixed precision (FP32 stencil arithmetic and multigrid; FP64 state, CG
# residual and stopping test, FP64 affine part of the state relation): every
# field within a stated relative error of the FP64 oracle.
# ---------------------------------------------------------------------------
MIXED_TOL = 1e-6


@pytest.mark.parametrize("case", ["blobs", "slot", "sphere"])
def test_mixed_precision_error_against_oracle(case):
    if case == "blobs":
        prm, geo, f = W.periodic_blobs(64)
        steps = 100
    elif case == "slot":
        prm, geo, f = W.slot_burner(64, 128)
        steps = 50
    else:
        prm, geo, f = W.sphere_burner(24)
        steps = 10
    prm["poisson_rtol"] = 1e-12
    prm["precision"] = W.MIXED
    pb, st = oracle_run(prm, geo, f, steps)
    sim = gpu_run(prm, geo, f, steps)
    worst = compare(sim, oracle_fields(pb, st), MIXED_TOL)
    print(case, {k: f"{v:.2e}" for k, v in worst.items()})


def test_slot_burner_full_size_mixed_matches_oracle():
    """The bench's headline configuration: 256x512, mixed precision,
    poisson_rtol = 1e-10, graphs on, 4 steps (two of them through the step
    graph).  Scalars to 1e-9; P, v and F to the mixed-precision bound."""
    prm, geo, f = W.slot_burner()
    prm["precision"] = W.MIXED
    pb, st = oracle_run(prm, geo, f, 4)
    sim = gpu_run(prm, geo, f, 4)
    ref = oracle_fields(pb, st)
    compare(sim, ref, 1e-9, names=["Z", "H", "T", "RHO", "KAPPA"])
    compare(sim, ref, MIXED_TOL, names=["U", "V", "P", "FX", "FY"])
    assert sim.query(7) <= 1e-10 and sim.query(6) <= 1e-10


def test_sphere_burner_full_size_mixed_matches_oracle():
    """The 3D configuration the bench times with --config sphere: 192^3,
    mixed precision, poisson_rtol = 1e-10, one step (the oracle takes about
    20 s and 4 GB for it).  Every field to the mixed-precision bound."""
    prm, geo, f = W.sphere_burner(192)
    prm["precision"] = W.MIXED
    pb, st = oracle_run(prm, geo, f, 1)
    sim = gpu_run(prm, geo, f, 1)
    compare(sim, oracle_fields(pb, st), MIXED_TOL)
    assert np.array_equal(sim.get("CHI"), V(pb.ibm["chi"], pb.g))
    assert sim.query(7) <= 1e-10 and sim.query(6) <= 1e-10


# ---------------------------------------------------------------------------
# The parity bar at full size: the bench's 256x512 slot burner over 100 steps
# (FP64 within 1e-9 on every field; mixed precision within its stated bound)
# and the 192^3 sphere burner in FP64.  The oracle's 100 slot steps are shared.
# ---------------------------------------------------------------------------
_FULL = {}


def _slot_full_oracle():
    if "slot" not in _FULL:
        prm, geo, f = W.slot_burner()
        prm["poisson_rtol"] = 1e-13
        _FULL["slot"] = oracle_run(prm, geo, f, 100)
    return _FULL["slot"]


def test_slot_burner_full_size_100_steps_fp64_within_1e9():
    prm, geo, f = W.slot_burner()
    prm["poisson_rtol"] = 1e-13
    pb, st = _slot_full_oracle()
    sim = gpu_run(prm, geo, f, 100)
    worst = compare(sim, oracle_fields(pb, st), 1e-9)
    print("slot 256x512 fp64 100 steps", {k: f"{v:.1e}" for k, v in worst.items()})
    sim.close()


def test_slot_burner_full_size_100_steps_mixed_within_bound():
    prm, geo, f = W.slot_burner()
    prm["poisson_rtol"] = 1e-12
    prm["precision"] = W.MIXED
    pb, st = _slot_full_oracle()
    sim = gpu_run(prm, geo, f, 100)
    worst = compare(sim, oracle_fields(pb, st), MIXED_TOL)
    print("slot 256x512 mixed 100 steps", {k: f"{v:.1e}" for k, v in worst.items()})
    sim.close()


def test_sphere_burner_full_size_fp64_within_1e9():
    """192^3 in FP64, 3 steps (one eager start-up step and two through the step
    graph); the oracle takes about 10 s and 4 GB per step."""
    prm, geo, f = W.sphere_burner(192)
    prm["poisson_rtol"] = 1e-13
    pb, st = oracle_run(prm, geo, f, 3)
    sim = gpu_run(prm, geo, f, 3)
    worst = compare(sim, oracle_fields(pb, st), 1e-9)
    print("sphere 192^3 fp64 3 steps", {k: f"{v:.1e}" for k, v in worst.items()})
    sim.close()


# ---------------------------------------------------------------------------
# Body given by surface markers: the marker-to-cell mask is integer work
# (bit-exact), S_m to rounding, then whole steps against the oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n,steps", [(2, 64, 10), (2, 96, 6), (3, 32, 4)])
def test_marker_body_matches_oracle(dim, n, steps):
    prm, geo, f = W.marker_burner(n, dim)
    prm["poisson_rtol"] = 1e-13
    pb, st = oracle_run(prm, geo, f, steps)
    sim = gpu_run(prm, geo, f, steps)
    assert np.array_equal(sim.get("CHI"), V(pb.ibm["chi"], pb.g))
    assert rel(sim.get("SM"), pb.ibm["Sm"]) < 1e-14
    worst = compare(sim, oracle_fields(pb, st), 1e-9)
    print("markers", dim, n, {k: f"{v:.1e}" for k, v in worst.items()})
    sim.close()


def test_marker_body_rejects_markers_denser_than_cells():
    from paper_2603_01727_gb300.lowmach import Simulation, SimError, SIM_EINVAL
    prm, geo, f = W.marker_burner(32, 2, spacing=0.3)
    with pytest.raises(SimError) as e:
        Simulation(prm, geo)
    assert e.value.status == SIM_EINVAL


# ---------------------------------------------------------------------------
# Per-step checks (sim_query): discrete continuity (Eq 3.24 with S_m), the
# global mass balance (text after Eq 4.22) and the predictor-corrector
# differences of Sec. 4.2.2
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("case,precision", [("slot", W.FP64), ("slot", W.MIXED), ("blobs", W.FP64),
                                            ("sphere", W.MIXED)])
def test_per_step_continuity_and_mass_balance(case, precision):
    from paper_2603_01727_gb300 import lowmach as LM
    if case == "slot":
        prm, geo, f = W.slot_burner(64, 128)
    elif case == "blobs":
        prm, geo, f = W.periodic_blobs(48)
    else:
        prm, geo, f = W.sphere_burner(32)
    prm["poisson_rtol"] = 1e-12
    prm["precision"] = precision
    sim = LM.Simulation(prm, geo)
    sim.set_fields(f)
    with pytest.raises(LM.SimError):
        sim.query(LM.SIM_Q_DIV_RESID)           # no step yet
    vol = float(np.prod(prm["L"][:prm["dim"]]))
    for k in range(6):
        sim.step(1)
        res = sim.query(LM.SIM_Q_DIV_RESID)
        scale = sim.query(LM.SIM_Q_DIV_SCALE)
        bal = sim.query(LM.SIM_Q_MASS_BALANCE)
        # the continuity residual is the pressure solve's residual: rtol-small
        assert res <= 1e-8 * max(scale, 1.0), (k, res, scale)
        # the outflow shift closes the global balance exactly (rounding only)
        assert abs(bal) <= 1e-12 * max(scale, 1.0) * vol, (k, bal, scale)
        assert sim.query(LM.SIM_Q_PC_DIFF_U) > 0.0 and sim.query(LM.SIM_Q_PC_DIFF_P) > 0.0
    sim.close()


def test_predictor_corrector_difference_matches_table2():
    """Taylor-Green vortex, 50x50, to t = 1.3: the L2 differences between
    predicted and corrected v1, v2 and P reproduce Table 2 (dt = 4e-3 and 2e-3)
    to 0.2 %, as the oracle does."""
    from conftest import golden
    from paper_2603_01727_gb300 import lowmach as LM
    rows = golden("taylor_green_table2.txt")
    want = {(float(r[1]), r[2]): float(r[3]) for r in rows}
    for dt in (4e-3, 2e-3):
        prm, geo, f = W.taylor_green(50, dt)
        sim = gpu_run(prm, geo, f, int(round(1.3 / dt)))
        got = {"P": sim.query(LM.SIM_Q_PC_DIFF_P), "v1": sim.query(LM.SIM_Q_PC_DIFF_U),
               "v2": sim.query(LM.SIM_Q_PC_DIFF_V)}
        for var, v in got.items():
            assert v == pytest.approx(want[(dt, var)], rel=2e-3), (dt, var, v, want[(dt, var)])
        sim.close()


# ---------------------------------------------------------------------------
# Execution paths and error handling
# ---------------------------------------------------------------------------
# ---------------------------------------------------------------------------
# Persistent 2D solve (one cooperative launch per pressure solve; opt-in,
# LOWMACH_PERSIST=1)
# ---------------------------------------------------------------------------
def _mixed_slot(nx, ny, steps, env, monkeypatch):
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    prm, geo, f = W.slot_burner(nx, ny)
    prm["precision"] = W.MIXED
    prm["poisson_rtol"] = 1e-12
    sim = gpu_run(prm, geo, f, steps)
    out = {k: sim.get(k) for k in ("U", "V", "Z", "RHO", "P")}
    its = (sim.query(4), sim.query(5))
    sim.close()
    for k in env:
        monkeypatch.delenv(k)
    return out, its


@pytest.mark.parametrize("nx,ny", [(64, 128), (256, 512), (96, 192)])
def test_persistent_solve_matches_the_kernel_chain(nx, ny, monkeypatch):
    """The persistent solve and the chain of level kernels run the same
    iteration; only the order of the block partial sums differs, so the fields
    agree to the solver tolerance and the iteration counts to one."""
    a, ia = _mixed_slot(nx, ny, 12, {"LOWMACH_PERSIST": "1"}, monkeypatch)
    b, ib = _mixed_slot(nx, ny, 12, {}, monkeypatch)
    for k in a:
        assert rel(a[k], b[k]) < 1e-9, (k, rel(a[k], b[k]))
    assert abs(ia[0] - ib[0]) <= 1 and abs(ia[1] - ib[1]) <= 1, (ia, ib)


def test_persistent_solve_graph_and_eager_agree_bitwise(monkeypatch):
    a, _ = _mixed_slot(64, 128, 9, {"LOWMACH_PERSIST": "1"}, monkeypatch)
    b, _ = _mixed_slot(64, 128, 9, {"LOWMACH_PERSIST": "1", "LOWMACH_NO_GRAPH": "1"}, monkeypatch)
    for k in a:
        assert np.array_equal(a[k], b[k]), k


def test_persistent_solve_barrier_timeout_is_reported(monkeypatch):
    """A barrier that waits for one block more than the grid has gives up
    after its poll limit: every block leaves, the step reports
    non-convergence, and the context stays usable for the next simulation."""
    from paper_2603_01727_gb300.lowmach import SimError, SIM_ENOCONV
    monkeypatch.setenv("LOWMACH_PERSIST", "1")
    monkeypatch.setenv("LOWMACH_PERSIST_TEST_TIMEOUT", "1")
    prm, geo, f = W.slot_burner(64, 128)
    prm["precision"] = W.MIXED
    with pytest.raises(SimError) as e:
        gpu_run(prm, geo, f, 1)
    assert e.value.status == SIM_ENOCONV
    monkeypatch.delenv("LOWMACH_PERSIST_TEST_TIMEOUT")
    sim = gpu_run(prm, geo, f, 2)
    assert sim.query(7) <= 1e-10
    sim.close()


@pytest.mark.parametrize("case,tile", [("slot", 16), ("slot", 64), ("sphere", 32)])
def test_stage_cell_tiles_change_nothing(case, tile):
    """The cell tile of the projection only changes which block computes a
    cell: the fields are bitwise those of the linear map."""
    if case == "slot":
        prm, geo, f = W.slot_burner(64, 128)
    else:
        prm, geo, f = W.sphere_burner(24)
    prm["precision"] = W.MIXED
    a = gpu_run(prm, geo, f, 5)
    b = gpu_run(dict(prm, stage_tile_x=tile), geo, f, 5)
    for k in ("U", "V", "Z", "H", "RHO", "P"):
        assert np.array_equal(a.get(k), b.get(k)), k
    a.close()
    b.close()


def test_graph_and_eager_paths_agree_bitwise(monkeypatch):
    prm, geo, f = W.slot_burner(32, 64)
    sim_g = gpu_run(prm, geo, f, 9)
    monkeypatch.setenv("LOWMACH_NO_GRAPH", "1")
    sim_e = gpu_run(prm, geo, f, 9)
    for k in ("U", "V", "Z", "P", "FY"):
        assert np.array_equal(sim_g.get(k), sim_e.get(k)), k


@pytest.mark.parametrize("case", ["slot", "sphere"])
def test_restart_blob_same_through_pinned_pageable_and_device_buffers(case):
    """sim_state_save / sim_state_load move the restart state as one
    contiguous image of the workspace's state arrays (padding zeroed at
    creation), into pinned or pageable host memory or device memory.  The three
    blobs must agree byte for byte, and a state loaded through either host
    buffer must step to the same bits."""
    import torch
    prm, geo, f = W.slot_burner(64, 128) if case == "slot" else W.sphere_burner(24)
    prm["precision"] = W.MIXED
    sim = gpu_run(prm, geo, f, 3)
    n = sim.state_size()
    pageable = np.zeros(n, dtype=np.uint8)
    pinned = torch.zeros(n, dtype=torch.uint8, pin_memory=True)
    device = torch.zeros(n, dtype=torch.uint8, device="cuda")
    sim.state_save(pageable)
    sim.state_save(pinned)
    sim.state_save(device)
    assert np.array_equal(pageable, pinned.numpy())
    assert np.array_equal(pageable, device.cpu().numpy())
    names = ("U", "V", "Z", "H", "P")
    sim.step(2)
    sim.sync()
    ref = {k: sim.get(k) for k in names}
    for blob in (pinned, pageable):
        sim.state_load(blob)
        sim.step(2)
        sim.sync()
        for k in names:
            assert np.array_equal(sim.get(k), ref[k]), k
    sim.close()


@pytest.mark.parametrize("case,buf", [("slot", "pinned"), ("slot", "pageable"), ("slot", "device"),
                                      ("sphere", "pinned"), ("sphere", "pageable"), ("sphere", "device")])
def test_step_save_equals_step_then_state_save(case, buf):
    """sim_step_save copies the arrays that are final after the corrector's
    state relation while the corrector's solve runs, the rest after the step:
    its blob must equal sim_step followed by sim_state_save byte for byte,
    through the eager first steps and the step graphs, into pinned or pageable
    host memory or device memory."""
    import torch
    from paper_2603_01727_gb300.lowmach import Simulation
    prm, geo, f = W.slot_burner(64, 128) if case == "slot" else W.sphere_burner(24)
    prm["precision"] = W.MIXED
    a, b = Simulation(prm, geo), Simulation(prm, geo)
    a.set_fields(f)
    b.set_fields(f)
    n = a.state_size()
    ref = np.zeros(n, dtype=np.uint8)
    if buf == "pinned":
        out = torch.zeros(n, dtype=torch.uint8, pin_memory=True)
    elif buf == "pageable":
        out = np.zeros(n, dtype=np.uint8)
    else:
        out = torch.zeros(n, dtype=torch.uint8, device="cuda")
    host = lambda o: o.cpu().numpy() if isinstance(o, torch.Tensor) else o
    for _ in range(5):
        a.step(1)
        a.state_save(ref)
        b.step_save(out)
        assert np.array_equal(ref, host(out))
    a.close()
    b.close()


def test_second_run_after_set_fields_repeats_the_first():
    """Setting the fields again restarts from level 0 whatever the previous
    run left in the rotating density buffers: after 5 steps (a count that is
    not a multiple of the three-level rotation) a second run on the same
    simulation reproduces the first bit for bit."""
    from paper_2603_01727_gb300.lowmach import Simulation
    prm, geo, f = W.slot_burner(32, 64)
    sim = Simulation(prm, geo)
    out = []
    for _ in range(2):
        sim.set_fields(f)
        sim.step(5)
        sim.sync()
        out.append({k: sim.get(k) for k in ("U", "V", "Z", "RHO", "P")})
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k]), k
    sim.close()


def test_warm_started_solves_match_oracle_and_restart(monkeypatch):
    """LOWMACH_EXTRAP=1: the pressure solves start from extrapolated guesses
    (2 P^n - P^(n-1); P* + P^n - P*^n).  Every solve still runs to its
    tolerance, so the fields stay within 1e-9 of the oracle.  The restart
    blob does not carry the guesses' history: a reloaded run takes plain
    guesses for two steps and agrees with the uninterrupted run to the
    solvers' tolerance."""
    monkeypatch.setenv("LOWMACH_EXTRAP", "1")
    prm, geo, f = W.slot_burner(64, 128)
    prm["poisson_rtol"] = 1e-13
    pb, st = oracle_run(prm, geo, f, 12)
    sim = gpu_run(prm, geo, f, 12)
    compare(sim, oracle_fields(pb, st), 1e-9)
    blob = np.zeros(sim.state_size(), dtype=np.uint8)
    sim.state_save(blob)
    sim.step(6)
    sim.sync()
    ref = {k: sim.get(k) for k in ("U", "V", "Z", "H", "P")}
    sim.state_load(blob)
    sim.step(6)
    sim.sync()
    for k, v in ref.items():
        assert rel(sim.get(k), v) <= 1e-10, k
    sim.close()


@pytest.mark.parametrize("case", ["slot", "sphere"])
def test_stencil_input_images_change_nothing(case, monkeypatch):
    """The mixed stage stencil reads float-float images of v, Z, H and kappa,
    split once per stage; LOWMACH_FF_IMAGES=0 splits each value as it is
    loaded.  Every value enters the stencil's arithmetic as the same
    float-float pair either way, so the runs agree bit for bit."""
    prm, geo, f = W.slot_burner(64, 128) if case == "slot" else W.sphere_burner(24)
    prm["precision"] = W.MIXED
    out = {}
    for img in ("1", "0"):
        monkeypatch.setenv("LOWMACH_FF_IMAGES", img)
        sim = gpu_run(prm, geo, f, 5)
        out[img] = {k: sim.get(k) for k in ("U", "V", "Z", "H", "P")}
        sim.close()
    for k in out["1"]:
        assert np.array_equal(out["1"][k], out["0"][k]), k


def test_repeat_runs_are_bitwise_deterministic():
    prm, geo, f = W.periodic_blobs(48)
    a = gpu_run(prm, geo, f, 12)
    b = gpu_run(prm, geo, f, 12)
    for k in ("U", "V", "Z", "P"):
        assert np.array_equal(a.get(k), b.get(k)), k


def test_nonconvergence_reported():
    from paper_2603_01727_gb300.lowmach import SimError, SIM_ENOCONV
    prm, geo, f = W.periodic_blobs(32)
    prm["poisson_max_iter"] = 1
    prm["poisson_rtol"] = 1e-14
    from paper_2603_01727_gb300.lowmach import Simulation
    sim = Simulation(prm, geo)
    sim.set_fields(f)
    sim.step(2)
    with pytest.raises(SimError) as e:
        sim.sync()
    assert e.value.status == SIM_ENOCONV


def test_nan_seeded_on_host_is_reported():
    from paper_2603_01727_gb300.lowmach import SimError, SIM_ENAN, Simulation
    prm, geo, f = W.periodic_blobs(32)
    f["Z"] = f["Z"].copy()
    f["Z"][5, 7] = np.nan
    sim = Simulation(prm, geo)
    sim.set_fields(f)
    sim.step(1)
    with pytest.raises(SimError) as e:
        sim.sync()
    assert e.value.status == SIM_ENAN


def test_unstable_penalisation_rejected():
    from paper_2603_01727_gb300.lowmach import SimError, SIM_EUNSTABLE, Simulation
    prm, geo, f = W.slot_burner(32, 64)
    prm["dt"] = 0.05                      # >= Re Da_ib = 0.02
    with pytest.raises(SimError) as e:
        Simulation(prm, geo)
    assert e.value.status == SIM_EUNSTABLE


def test_step_before_fields_is_a_state_error():
    from paper_2603_01727_gb300.lowmach import SimError, SIM_ESTATE, Simulation
    prm, geo, _ = W.periodic_blobs(16)
    sim = Simulation(prm, geo)
    with pytest.raises(SimError) as e:
        sim.step(1)
    assert e.value.status == SIM_ESTATE


@pytest.mark.parametrize("path", ["sweeps", "zmarch"])
@pytest.mark.parametrize("n,periodic_x,precision", [(48, False, W.MIXED), (48, False, W.FP64), (32, True, W.FP64),
                                                    (32, True, W.MIXED)])
def test_large_level_3d_multigrid_matches_cube_tiles(n, periodic_x, precision, path, monkeypatch):
    """The large-level 3D multigrid kernels -- the whole-level colour-sweep
    passes (default) and the z-marching ones (LOWMACH_MG3_SWEEPS=0) -- apply
    the same smoother, residual, restriction and prolongation as the
    cube-tile kernels (LOWMACH_MG3_TILES=1): same iteration counts and the
    same fields to solver tolerance, with every level on the kernels tested."""
    from paper_2603_01727_gb300.lowmach import SIM_Q_ITERS_PRED, SIM_Q_ITERS_CORR
    prm, geo, f = W.sphere_burner(n)
    prm["precision"] = precision
    prm["poisson_rtol"] = 1e-12
    if periodic_x:
        prm["bc"] = [[W.PERIODIC, W.PERIODIC]] + prm["bc"][1:]
    out = {}
    monkeypatch.setenv("LOWMACH_MG3_MIN_CELLS", "0")     # every level on the large-level kernels
    monkeypatch.setenv("LOWMACH_MG3_SWEEPS", "1" if path == "sweeps" else "0")
    for tiles in ("0", "1"):
        monkeypatch.setenv("LOWMACH_MG3_TILES", tiles)
        sim = gpu_run(prm, geo, f, 4)
        out[tiles] = ({k: sim.get(k) for k in ("U", "W", "Z", "P")},
                      (sim.query(SIM_Q_ITERS_PRED), sim.query(SIM_Q_ITERS_CORR)))
    assert out["0"][1] == out["1"][1], (out["0"][1], out["1"][1])
    for k in out["0"][0]:
        assert rel(out["0"][0][k], out["1"][0][k]) <= 1e-9, k


@pytest.mark.parametrize("n,periodic_x", [(48, False), (32, True)])
def test_3d_fast_diagonalisation_top_level_matches_vcycle_tail(n, periodic_x, monkeypatch):
    """Mixed precision in 3D solves the top coarse level (at most 4096 cells)
    exactly by fast diagonalisation; forcing the one-block V-cycle tail
    instead (an explicit tail size) must give the same fields to solver
    tolerance, with no more CG iterations for the exact coarse solve."""
    from paper_2603_01727_gb300.lowmach import (SIM_Q_ITERS_PRED, SIM_Q_ITERS_CORR, SIM_Q_TAIL_FDM, SIM_Q_TAIL_NX,
                                                SIM_Q_TAIL_NZ)
    prm, geo, f = W.sphere_burner(n)
    prm["precision"] = W.MIXED
    prm["poisson_rtol"] = 1e-12
    if periodic_x:
        prm["bc"] = [[W.PERIODIC, W.PERIODIC]] + prm["bc"][1:]
    out = {}
    for mode in ("fdm", "tail"):
        if mode == "tail":
            monkeypatch.setenv("LOWMACH_TAIL_CELLS", "4096")
        sim = gpu_run(prm, geo, f, 4)
        fdm = sim.query(SIM_Q_TAIL_FDM)
        assert fdm == (1.0 if mode == "fdm" else 0.0), (mode, fdm)
        if mode == "fdm":
            top = sim.query(SIM_Q_TAIL_NX)
            assert sim.query(SIM_Q_TAIL_NZ) == top and top ** 3 <= 4096, top
        out[mode] = ({k: sim.get(k) for k in ("U", "W", "Z", "P")},
                     sim.query(SIM_Q_ITERS_PRED) + sim.query(SIM_Q_ITERS_CORR))
        sim.close()
    assert out["fdm"][1] <= out["tail"][1], (out["fdm"][1], out["tail"][1])
    for k in out["fdm"][0]:
        assert rel(out["fdm"][0][k], out["tail"][0][k]) <= 1e-9, k


@pytest.mark.parametrize("case,precision", [("slot", W.MIXED), ("slot", W.FP64), ("sphere", W.MIXED)])
def test_cg_iterations_captured_ahead_of_the_loop_change_nothing(case, precision, monkeypatch):
    """A graph-launched solve captures its first CG iterations ahead of its
    while node; once a solve has converged, the remaining captured iterations
    must leave x and the reported scalars untouched (the update kernels test
    the done flag).  A prefix longer than any solve (40 iterations) and none
    must give bitwise the same fields and iteration counts, through the eager
    first steps and the step graphs."""
    from paper_2603_01727_gb300.lowmach import SIM_Q_ITERS_PRED, SIM_Q_ITERS_CORR, SIM_Q_KERNEL_LAUNCHES, Simulation
    prm, geo, f = W.slot_burner(64, 128) if case == "slot" else W.sphere_burner(24)
    prm["precision"] = precision
    out = {}
    for u in ("40", "0"):
        monkeypatch.setenv("LOWMACH_CG_PREFIX", u)
        sim = Simulation(prm, geo)
        sim.set_fields(f)
        its = []
        for _ in range(5):
            sim.step(1)
            its.append((sim.query(SIM_Q_ITERS_PRED), sim.query(SIM_Q_ITERS_CORR)))
        launches = sim.query(SIM_Q_KERNEL_LAUNCHES)
        out[u] = ({k: sim.get(k) for k in ("U", "V", "Z", "H", "P")}, its, launches)
        sim.close()
    assert out["40"][1] == out["0"][1], (out["40"][1], out["0"][1])
    assert all(a < 40 and b < 40 for a, b in out["0"][1])
    for k in out["0"][0]:
        assert np.array_equal(out["40"][0][k], out["0"][0][k]), k
    # the captured iterations are launched whether or not they were needed
    assert out["40"][2] > out["0"][2], (out["40"][2], out["0"][2])


@pytest.mark.parametrize("case", ["slot", "sphere"])
def test_mixed_state_relation_is_fp64_accurate(case):
    """The mixed path's state relation evaluates kappa = T^0.7 with a
    float-float correction of an FP32 seed and rho = p0 / T with FP32
    reciprocal steps and one FP64 Newton step; both must match the FP64
    formulas of the stored T far below the FP32 rounding (~6e-8) they replace.
    Bounds: kappa's correction delta = T^7 / y0^10 - 1 comes from eight
    float-float products and a quotient, each ~2^-46 relative, so delta is
    good to ~1e-13 and kappa = y0 (1 + delta/10 + ...) to ~1e-14; one FP64
    Newton step from a seed within ~2^-24 leaves ~2^-48 (plus rounding)."""
    from paper_2603_01727_gb300.lowmach import SIM_Q_P0
    if case == "slot":
        prm, geo, f = W.slot_burner(64, 128)
    else:
        prm, geo, f = W.sphere_burner(24)
    prm["precision"] = W.MIXED
    sim = gpu_run(prm, geo, f, 3)
    T = sim.get("T")
    kap = sim.get("KAPPA")
    rho = sim.get("RHO")
    p0 = sim.query(SIM_Q_P0)
    assert np.all(T > 0.0)
    ek = np.max(np.abs(kap / T ** 0.7 - 1.0))
    er = np.max(np.abs(rho * T / p0 - 1.0))
    assert ek < 1e-13, ek          # measured 2e-14; an FP32 kappa would be ~6e-8
    assert er < 1e-14, er          # measured 3.6e-15
    sim.close()


def test_adjoint_gradient_matches_the_oracles_complex_step_derivative():
    """The GPU adjoint's gradient of the heat-release objective against the
    oracle's own derivative of it, taken by the complex step (exact to
    rounding, no difference error): slot burner 24x48 whose profile is a sum
    of 6 Gaussian bumps, 6 steps.  Every component and the derivative along
    a random direction within 1e-6 relative (the bar for gradients); the
    objective values agree to 1e-9."""
    from oracle import objective as O
    from paper_2603_01727_gb300.adjoint import HeatReleaseProblem
    from test_gpu_adjoint import _case, _direction
    prm, geo, f, A, c = _case(24, 48, 6, 32)
    N = 6
    pb = HeatReleaseProblem(prm, geo, f, A, nsteps=N, every=3)
    Jg = pb.value(c)
    gc, _ = pb.gradient()
    pb.close()

    def J(cc):
        p = S.Problem(prm, dict(geo, profile=list(A @ cc)))
        st = S.initial_state(p, f["v"], f["Z"], f["H"])
        return O.objective(p, st, N, S.advance)

    assert abs(J(c) - Jg) <= 1e-9 * abs(Jg)
    g_cs = np.array([O.complex_step_derivative(J, c, d) for d in np.eye(len(c))])
    gc = np.asarray(gc, dtype=float)
    err = float(np.max(np.abs(gc - g_cs)) / np.max(np.abs(g_cs)))
    e = _direction(len(c), seed=5)
    cs_e = O.complex_step_derivative(J, c, e)
    err_e = abs(float(gc @ e) - cs_e) / abs(cs_e)
    print("adjoint vs oracle complex step: components %.1e, direction %.1e" % (err, err_e))
    assert err <= 1e-6 and err_e <= 1e-6, (err, err_e)
