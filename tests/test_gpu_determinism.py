"""Run-to-run reproducibility of a step on the GPU.

Every sum that many threads add into (energies, gradient, Hessian blocks, the preconditioner diagonal, the
Dirichlet term, the coarse matrix) is accumulated exactly in integer fixed point, and the lists built with
atomic appends (contact pairs, contact incidences, ABD coupling blocks) are put into a canonical order, so
the same step from the same state with the same PCG launch shape gives the same bits: positions, velocities,
affine-body coordinates and the solver statistics."""
import numpy as np
import pytest

from paper_2609_25653_b300 import scenes

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _run(sc, n, precision=None, batch=None, **kw):
    from paper_2609_25653_b300 import ipcsim
    args = dict(kw)
    if precision is not None:
        args["precision"] = precision
    sim = ipcsim.Simulator.batch(batch, **args) if batch else ipcsim.Simulator(sc, **args)
    stats = []
    for _ in range(n):
        st = sim.step()
        assert st["status"] == 0
        stats.append((st["newton_iters"], st["pcg_iters_total"], st["n_pairs_max"], st["ls_halvings"],
                      st["energy_end"]))
    x, v, q, qd = sim.get_state()
    sim.close()
    return x, v, q, qd, stats


def _same(a, b):
    for u, w in zip(a[:4], b[:4]):
        assert u.shape == w.shape and np.array_equal(u.view(np.uint64), w.view(np.uint64))
    assert a[4] == b[4]


@pytest.mark.parametrize("mixed", [False, True])
def test_grasp_steps_are_bit_identical(mixed):
    """The reduced arm-gripper grasp through contact onset and squeeze (friction, stitches, the ABD object)."""
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.arm_gripper_grasp_reduced(0, n_steps=10)
    prec = ipcsim.PREC_MIXED if mixed else ipcsim.PREC_FP64
    a = _run(sc, 10, prec)
    b = _run(sc, 10, prec)
    assert max(s[2] for s in a[4]) > 20  # contacts were active
    _same(a, b)


def test_batch_and_joints_are_bit_identical():
    scs = [scenes.jointed_arm(3, n_steps=6), scenes.fingertip_press(0, n_steps=6)]
    a = _run(None, 6, batch=scs)
    b = _run(None, 6, batch=scs)
    _same(a, b)
    c = _run(scs[0], 6)
    d = _run(scs[0], 6)
    _same(c, d)


def test_restarted_step_is_bit_identical():
    """Setting the state back and stepping again reproduces the step exactly (the pair capacity, trees and
    lists the first pass left behind do not change the result)."""
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.arm_gripper_grasp_reduced(0, n_steps=8)
    sim = ipcsim.Simulator(sc)
    for _ in range(5):
        sim.step()
    s0 = sim.get_state()
    sim.step()
    s1 = sim.get_state()
    sim.set_state(*s0)
    sim.set_kinematic(sc["kin_T"][5])
    sim.step_index = 5
    sim.step()
    s2 = sim.get_state()
    for u, w in zip(s1, s2):
        assert np.array_equal(u.view(np.uint64), w.view(np.uint64))
