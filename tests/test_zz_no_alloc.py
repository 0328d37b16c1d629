"""sim_poisson_solve_noalloc: the pressure solve for callers that cannot
allocate device memory (a plug-in inside an application that owns all device
memory, a fixed memory budget, a loop that cannot take cudaMalloc's implicit
synchronisation).  It uses the library's static device scratch instead of a
workspace; its results must match the workspace entry point's.

Collected last (file name) so that a run stopping at the first failure has
already run every other test."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2603_01727_gb300 import build
    build.build()


def _solve_both(torch, n, periodic, seed):
    from paper_2603_01727_gb300.lowmach import poisson_solve, poisson_solve_noalloc
    rng = np.random.Generator(np.random.PCG64(seed))
    h = [1.0 / n[d] * (1.0 + 0.25 * d) for d in range(len(n))]
    b = torch.tensor(rng.normal(size=tuple(reversed(n))), dtype=torch.float64, device="cuda")
    P_ws = torch.zeros_like(b)
    P_na = torch.zeros_like(b)
    it_ws, rr_ws = poisson_solve(b, P_ws, h, periodic, rtol=1e-12, max_iter=300)
    it_na, rr_na = poisson_solve_noalloc(b, P_na, h, periodic, rtol=1e-12, max_iter=300)
    return (it_ws, rr_ws, P_ws.cpu().numpy()), (it_na, rr_na, P_na.cpu().numpy())


def test_noalloc_solve_matches_workspace_solve_on_consecutive_calls():
    import torch
    assert torch.cuda.is_available(), "GPU test"
    # two calls in a row on different grids: the second call starts from the
    # scratch contents the first one left behind
    for n, periodic, seed in (((64, 64), (1, 1), 3), ((96, 40), (0, 0), 4)):
        (it_ws, rr_ws, P_ws), (it_na, rr_na, P_na) = _solve_both(torch, n, periodic, seed)
        assert rr_na <= 1e-12 and rr_ws <= 1e-12
        scale = float(np.max(np.abs(P_ws)))
        assert float(np.max(np.abs(P_na - P_ws))) <= 1e-9 * scale, (n, it_ws, it_na)
        assert it_na == it_ws


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2603_01727_gb300.lowmach import SimError, SIM_ENOMEM, poisson_solve_noalloc
    b = torch.zeros((1024, 1024), dtype=torch.float64, device="cuda")   # ~40 MiB of scratch needed
    P = torch.zeros_like(b)
    with pytest.raises(SimError) as e:
        poisson_solve_noalloc(b, P, (1e-3, 1e-3), (1, 1))
    assert e.value.status == SIM_ENOMEM
