"""Batched pressure solves (sim_poisson_solve_batch): nb independent systems
on one 2D grid advanced by one launch per multigrid level and CG update.
Every system must get exactly the iterates it gets when solved alone (the
per-system arithmetic and block decomposition are those of a single solve),
so the comparison is bitwise, iteration counts included; and the answers
match the exact transform solve of the oracle."""

import numpy as np
import pytest

from oracle import poisson as OP
from oracle.operators import Grid

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_01727_gb300 import build
    build.build()


def _systems(nb, n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    b = rng.normal(size=(nb, n[1], n[0]))
    b *= 10.0 ** rng.uniform(-2, 2, size=(nb, 1, 1))       # uneven scales: uneven iteration counts
    x0 = rng.normal(size=(nb, n[1], n[0])) * 1e-3
    return b, x0


@pytest.mark.parametrize("n,periodic", [((64, 128), (1, 0)), ((96, 40), (0, 0)), ((48, 48), (1, 1))])
@pytest.mark.parametrize("precision", [0, 1])
def test_batched_solve_is_bitwise_the_single_solve(n, periodic, precision):
    import torch
    from paper_2603_01727_gb300.lowmach import poisson_solve_batch
    nb = 5
    b, x0 = _systems(nb, n, 3)
    h = (1.0 / n[0], 2.0 / n[1])
    bt = torch.tensor(b, device="cuda", dtype=torch.float64)
    Pb = torch.tensor(x0, device="cuda", dtype=torch.float64)
    its, rrs = poisson_solve_batch(bt, Pb, h, periodic, precision=precision, rtol=1e-11, max_iter=300)
    for k in range(nb):
        P1 = torch.tensor(x0[k:k + 1], device="cuda", dtype=torch.float64)
        it1, rr1 = poisson_solve_batch(bt[k:k + 1].contiguous(), P1, h, periodic, precision=precision,
                                       rtol=1e-11, max_iter=300)
        assert its[k] == it1[0], (k, its[k], it1[0])
        assert rrs[k] == rr1[0]
        assert torch.equal(Pb[k], P1[0]), k
        assert rrs[k] <= 1e-11


def test_batched_solve_matches_transform_solve_and_single_fp64_path():
    import torch
    from paper_2603_01727_gb300.lowmach import poisson_solve_batch, poisson_solve
    n, periodic = (64, 32), (1, 0)
    nb = 3
    b, _ = _systems(nb, n, 7)
    g = Grid(n, (1.0, 0.5))
    bt = torch.tensor(b, device="cuda", dtype=torch.float64)
    Pb = torch.zeros_like(bt)
    poisson_solve_batch(bt, Pb, g.h, periodic, rtol=1e-13, max_iter=300)
    for k in range(nb):
        ref = OP.solve(b[k], g, periodic)
        err = float(np.max(np.abs(Pb[k].cpu().numpy() - ref)) / np.max(np.abs(ref)))
        assert err < 1e-9, (k, err)
        P1 = torch.zeros_like(bt[k])
        poisson_solve(bt[k].contiguous(), P1, g.h, periodic, rtol=1e-13, max_iter=300)
        assert torch.equal(P1, Pb[k])            # the nb = 1 path is the stand-alone solve


def test_batched_solve_rejects_3d_free_sizes():
    from paper_2603_01727_gb300.lowmach import load, SIM_EINVAL
    import ctypes
    lib = load()
    sz = ctypes.c_size_t()
    n = (ctypes.c_int * 2)(7, 9)                  # does not coarsen: one level
    per = (ctypes.c_int * 2)(0, 0)
    assert lib.sim_poisson_batch_workspace_size(n, per, 4, 0, ctypes.byref(sz)) == SIM_EINVAL
    n2 = (ctypes.c_int * 2)(64, 64)
    assert lib.sim_poisson_batch_workspace_size(n2, per, 0, 0, ctypes.byref(sz)) == SIM_EINVAL
