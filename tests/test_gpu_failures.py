"""Host-made failures of a step: every failed sim_step leaves the state at the start of that step, reports
its status in the step statistics, and leaves the simulator usable (no GPU fault is involved: the failures
come from the inputs or from limits set on the host)."""
import math

import numpy as np
import pytest

from paper_2609_25653_b300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

IPC_ERR_NAN, IPC_ERR_NEWTON_MAXIT, IPC_ERR_CAPACITY = -7, -4, -10


def _sim(sc, **kw):
    from paper_2609_25653_b300 import ipcsim
    return ipcsim.Simulator(sc, **kw)


def _state(sim):
    x, v, q, qd = sim.get_state()
    return [a.copy() for a in (x, v, q, qd)]


def _same(a, b):
    return all(np.array_equal(u, w) for u, w in zip(a, b))


def test_nan_transform_fails_and_restores_state():
    """A non-finite kinematic target is refused before the step starts (IPC_ERR_ARG)."""
    sc = scenes.fingertip_press(0, n_steps=4)
    sim = _sim(sc)
    sim.step()
    before = _state(sim)
    T = sc["kin_T"][2].copy()
    T[1, 2, 3] = math.nan  # the plate's target height
    st = sim.step(T, raise_on_error=False)
    assert st["status"] == -1
    assert _same(before, _state(sim))
    assert sim.step_index == 1
    # the simulator is still usable: the proper transform steps normally
    st = sim.step()
    assert st["status"] == 0 and st["min_dist"] > 0


def test_poisoned_barrier_stiffness_fails_and_restores_state():
    sc = scenes.fingertip_press(0, n_steps=4)
    sim = _sim(sc, kappa=math.inf)
    before = _state(sim)
    st = sim.step(raise_on_error=False)
    assert st["status"] == IPC_ERR_NAN
    assert _same(before, _state(sim))


def test_pcg_budget_is_reported_as_unconverged():
    sc = scenes.fingertip_press(0, n_steps=4)
    sim = _sim(sc, max_pcg=1, max_newton=3)
    before = _state(sim)
    st = sim.step(raise_on_error=False)
    assert st["pcg_unconverged"] > 0
    assert st["pcg_iters_max"] <= 1
    if st["status"] != 0:
        assert st["status"] == IPC_ERR_NEWTON_MAXIT
        assert _same(before, _state(sim))


def test_pair_capacity_limit_fails_and_restores_state():
    """A pair buffer limit below what the step needs: IPC_ERR_CAPACITY, state at x_t."""
    from oracle import ipc as orc
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.abd_box_drop(n_steps=6)  # the box lands during the first step: more pairs than at x0
    ref = _sim(sc)
    S = orc.Scene(sc)
    x0 = torch.as_tensor(np.ascontiguousarray(S.positions(S.z0)), device="cuda")
    n0 = ref.active_pairs(x0)[0].shape[0]
    st = ref.step()
    assert st["n_pairs_max"] > n0 > 0, (n0, st["n_pairs_max"])
    sim = _sim(sc, pair_capacity=n0, pair_capacity_max=n0)
    before = _state(sim)
    st = sim.step(raise_on_error=False)
    assert st["status"] == IPC_ERR_CAPACITY
    assert _same(before, _state(sim))
    with pytest.raises(ipcsim.IpcError) as e:
        sim.step()
    assert e.value.code == IPC_ERR_CAPACITY
