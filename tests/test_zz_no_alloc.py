"""The allocation-free barrier entry point gives the same result as sim_eval_barrier.

Some callers cannot allocate device memory once they run (a control loop on
a fixed memory budget, or a process whose device memory belongs to another
allocator); sim_eval_barrier_noalloc serves them from a static device array.
This file is collected last so that a run stopping at the first failure has
run every other test before it."""
import numpy as np
import pytest

from paper_2609_25653_b300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_barrier_matches_allocating_entry_point_twice():
    from oracle import ipc as orc
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.fingertip_press(1)
    S = orc.Scene(sc)
    X = sc["fem_X"].copy()
    X[:, 2] = 0.5e-3 + (X[:, 2] - 0.5e-3) * 0.96 - 0.35e-3
    z = S.z0.copy()
    z[:S.n_fem_dof] = X.reshape(-1)
    xv = S.positions(z)
    xv[S.nf + S.na_v + 8:] += np.array([0, 0, -0.45e-3])
    sim = ipcsim.Simulator(sc)
    x_dev = torch.as_tensor(xv, device="cuda")
    rec, _ = sim.active_pairs(x_dev)
    n = rec.shape[0]
    assert n > 10
    E_ref, g_ref, H_ref = sim.eval_barrier(x_dev, rec, project=True)
    # outputs allocated once, before the calls; every call starts from garbage in them
    E = torch.empty((1,), dtype=torch.float64, device="cuda")
    g = torch.empty((sim.n_nodes, 3), dtype=torch.float64, device="cuda")
    H = torch.empty((n, 12, 12), dtype=torch.float64, device="cuda")
    rec = rec.contiguous()
    free_after = []
    for call in range(2):
        for t in (E, g, H):
            t.fill_(7.0)
        torch.cuda.synchronize()
        sim.eval_barrier_noalloc(x_dev, rec, E, g, H, project=True)
        torch.cuda.synchronize()
        # the first call may load the library's device code (and the static array) onto the device;
        # from then on no call changes the device's free memory
        free_after.append(torch.cuda.mem_get_info()[0])
        assert abs(E.item() - E_ref.item()) <= 1e-12 * abs(E_ref.item())
        assert torch.max(torch.abs(g - g_ref)).item() <= 1e-12 * torch.max(torch.abs(g_ref)).item()
        assert torch.max(torch.abs(H - H_ref)).item() <= 1e-12 * torch.max(torch.abs(H_ref)).item()
    # a third call, with nothing else between the two readings, allocates nothing
    torch.cuda.synchronize()
    before = torch.cuda.mem_get_info()[0]
    sim.eval_barrier_noalloc(x_dev, rec, E, g, H, project=True)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == before
