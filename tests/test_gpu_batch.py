"""Batched flames (sim_batch_*): independent simulations of uneven sizes
advanced by one CUDA graph per step.  A batch must give bit-for-bit the
result of stepping each simulation on its own, and its members keep their
parity with the FP64 oracle."""

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


def _flames(precision):
    out = []
    for (nx, ny), Re, zst, ratio in (((32, 64), 120.0, 0.05, 6.0), ((48, 96), 300.0, 0.07, 4.5),
                                     ((64, 128), 200.0, 0.055, 7.5)):
        prm, geo, f = W.slot_burner(nx, ny, Re=Re, Z_st=zst, density_ratio=ratio, Da_ib=max(1e-4, (2.0 / nx) ** 2))
        prm["precision"] = precision
        prm["poisson_rtol"] = 1e-12
        out.append((prm, geo, f))
    return out


def _sims(flames, stream):
    from paper_2603_01727_gb300.lowmach import Simulation
    sims = []
    for prm, geo, f in flames:
        s = Simulation(prm, geo, stream=stream)
        s.set_fields(f)
        sims.append(s)
    return sims


@pytest.mark.parametrize("precision", [W.FP64, W.MIXED])
def test_batch_is_bitwise_equal_to_separate_steps(precision):
    import torch
    from paper_2603_01727_gb300.lowmach import Batch
    flames = _flames(precision)
    stream = torch.cuda.Stream()
    alone = _sims(flames, stream)
    for s in alone:
        s.step(9)                        # eager steps, then every rotation phase of the graphs
        s.sync()
    members = _sims(flames, stream)
    batch = Batch(members, stream=stream)
    batch.step(4)
    batch.step(5)
    batch.sync()
    for a, b in zip(alone, members):
        names = ["U", "V", "Z", "H", "T", "RHO", "P", "FX", "FY"]
        for k in names:
            assert np.array_equal(a.get(k), b.get(k)), k


def _same_grid_flames(precision):
    """Four flames on one 64x128 grid (one batched-solve group) with different
    Re, Z_st and density ratio, and one 32x64 flame solved on its own."""
    out = []
    for (nx, ny), Re, zst, ratio in (((64, 128), 150.0, 0.05, 6.0), ((64, 128), 300.0, 0.07, 4.5),
                                     ((64, 128), 220.0, 0.06, 7.5), ((32, 64), 120.0, 0.055, 7.0),
                                     ((64, 128), 80.0, 0.045, 5.0)):
        prm, geo, f = W.slot_burner(nx, ny, Re=Re, Z_st=zst, density_ratio=ratio, Da_ib=max(1e-4, (2.0 / nx) ** 2))
        prm["precision"] = precision
        prm["poisson_rtol"] = 1e-12
        out.append((prm, geo, f))
    return out


@pytest.mark.parametrize("precision", [W.FP64, W.MIXED])
def test_batched_solves_are_bitwise_equal_to_separate_steps(precision):
    """Same-grid members share one batched pressure solve per stage; every
    member must still get bitwise its own result."""
    import torch
    from paper_2603_01727_gb300.lowmach import Batch, SIM_Q_ITERS_PRED, SIM_Q_ITERS_CORR
    flames = _same_grid_flames(precision)
    stream = torch.cuda.Stream()
    alone = _sims(flames, stream)
    for s in alone:
        s.step(9)
        s.sync()
    members = _sims(flames, stream)
    batch = Batch(members, stream=stream)
    assert batch.workspace is not None             # a batched-solve group exists
    batch.step(4)
    batch.step(5)
    batch.sync()
    assert batch.launches() > 0
    for a, b in zip(alone, members):
        for k in ["U", "V", "Z", "H", "T", "RHO", "P", "FX", "FY"]:
            assert np.array_equal(a.get(k), b.get(k)), k
        for q in (SIM_Q_ITERS_PRED, SIM_Q_ITERS_CORR):
            assert a.query(q) == b.query(q)


def test_batch_without_batched_solves_matches_batched():
    import torch
    from paper_2603_01727_gb300.lowmach import Batch
    flames = _same_grid_flames(W.MIXED)
    stream = torch.cuda.Stream()
    out = []
    for batched in (True, False):
        members = _sims(flames, stream)
        batch = Batch(members, stream=stream, batched_solves=batched)
        batch.step(7)
        batch.sync()
        out.append([m.get("P") for m in members])
        batch.close()
    for a, b in zip(*out):
        assert np.array_equal(a, b)


def test_batch_member_matches_oracle():
    import torch
    from paper_2603_01727_gb300.lowmach import Batch
    flames = _flames(W.FP64)
    stream = torch.cuda.Stream()
    members = _sims(flames, stream)
    batch = Batch(members, stream=stream)
    batch.step(6)
    batch.sync()
    prm, geo, f = flames[1]
    pb = S.Problem(prm, geo)
    st = S.initial_state(pb, f["v"], f["Z"], f["H"])
    for _ in range(6):
        st = S.advance(pb, st)
    g = pb.g
    ref = {"U": V(st.v[0], g), "V": V(st.v[1], g), "Z": V(st.Z, g), "T": V(st.T, g), "P": V(st.P, g)}
    for k, r in ref.items():
        err = float(np.max(np.abs(members[1].get(k) - r)) / np.max(np.abs(r)))
        assert err <= 1e-9, (k, err)


def test_batch_requires_lockstep():
    import torch
    from paper_2603_01727_gb300.lowmach import Batch, SimError, SIM_ESTATE
    flames = _flames(W.MIXED)[:2]
    stream = torch.cuda.Stream()
    members = _sims(flames, stream)
    members[0].step(3)
    members[1].step(4)
    members[0].sync()
    members[1].sync()
    batch = Batch(members, stream=stream)
    with pytest.raises(SimError) as e:
        batch.step(1)
    assert e.value.status == SIM_ESTATE


def test_autotuner_picks_a_measured_candidate():
    from paper_2603_01727_gb300 import autotune
    prm, geo, f = _flames(W.MIXED)[0]
    best, table = autotune.tune(prm, geo, f, candidates=((2, 0), (1, 0)), copies=2)
    assert best in table and all(t > 0 for t in table.values())
    assert table[best] == min(table.values())


@pytest.mark.parametrize("precision", [W.FP64, W.MIXED])
def test_member_batched_stage_kernels_are_bitwise_equal_to_separate_steps(precision):
    """Two solve groups of different grids (2 x 32x64, 3 x 48x96): every stage
    kernel of the five members runs as one launch over a work list that spans
    both grid sizes; each member keeps its own block decomposition, so the
    batch still gives the separate steps bit for bit."""
    import torch
    from paper_2603_01727_gb300.lowmach import Batch
    flames = []
    for (nx, ny), Re, zst, ratio in (((32, 64), 120.0, 0.05, 6.0), ((48, 96), 300.0, 0.07, 4.5),
                                     ((32, 64), 90.0, 0.06, 7.0), ((48, 96), 150.0, 0.045, 5.5),
                                     ((48, 96), 220.0, 0.065, 6.5)):
        prm, geo, f = W.slot_burner(nx, ny, Re=Re, Z_st=zst, density_ratio=ratio, Da_ib=max(1e-4, (2.0 / nx) ** 2))
        prm["precision"] = precision
        prm["poisson_rtol"] = 1e-12
        flames.append((prm, geo, f))
    stream = torch.cuda.Stream()
    alone = _sims(flames, stream)
    for s in alone:
        s.step(9)
        s.sync()
    members = _sims(flames, stream)
    batch = Batch(members, stream=stream)
    batch.step(9)
    batch.sync()
    assert batch.launches() > 0
    for a, b in zip(alone, members):
        for k in ("U", "V", "Z", "H", "T", "RHO", "P", "FX", "FY"):
            assert np.array_equal(a.get(k), b.get(k)), k
