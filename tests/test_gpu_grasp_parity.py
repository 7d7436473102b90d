"""Oracle parity on reduced versions of the benchmarked scenes.

The arm-gripper grasp at reduced resolution keeps every ingredient of the benchmarked scene: seven kinematic
arm links on the seeded joint wobble, two kinematic finger bases with stitched fin-ray fingertips, the ABD
ellipsoid on the ground quad, friction mu = 0.6.  The soft-gripper squeeze keeps its deformable cylinder.
The CPU oracle runs each whole (short) trajectory; the CUDA path then starts from the oracle's state at
sampled steps spanning contact onset, squeeze, hold and lift (teacher forcing) and must reach the oracle's
next state: within 1e-8 of the bounding-box diagonal in FP64, 1e-5 in mixed precision.  Every launch shape
the PCG autotuner may pick, and the operator streamed from global memory instead of staged in shared
memory, must give the FP64 result too."""
import numpy as np
import pytest

from paper_2609_25653_b300 import scenes
from tests.conftest import oracle_trajectory

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PARITY = dict(newton_tol=1e-9, pcg_rtol=1e-12)


@pytest.fixture(scope="module")
def grasp():
    sc = scenes.arm_gripper_grasp_reduced(0, n_steps=16, **PARITY)
    S, states = oracle_trajectory(sc)
    return sc, S, states


@pytest.fixture(scope="module")
def cylinder():
    sc = scenes.soft_gripper_cylinder_reduced(0, n_steps=12, **PARITY)
    S, states = oracle_trajectory(sc)
    return sc, S, states


def _sim(sc, **kw):
    from paper_2609_25653_b300 import ipcsim
    return ipcsim.Simulator(sc, **kw)


def _teacher_forced_step(sim, sc, S, states, k):
    """One GPU step from the oracle's state at step k; error against the oracle's state at k + 1."""
    nfd, nab = S.n_fem_dof, S.nab
    z, zd = states[k]
    sim.set_state(z[:nfd].reshape(-1, 3), zd[:nfd].reshape(-1, 3),
                  z[nfd:nfd + 12 * nab].reshape(-1, 12) if nab else None,
                  zd[nfd:nfd + 12 * nab].reshape(-1, 12) if nab else None)
    sim.set_kinematic(sc["kin_T"][k])
    sim.step_index = k
    st = sim.step()
    assert st["status"] == 0 and st["min_dist"] > 0
    xg, _, qg, _ = sim.get_state()
    zn = states[k + 1][0]
    err = np.max(np.abs(xg - zn[:nfd].reshape(-1, 3))) / S.L
    if nab:
        qo = zn[nfd:nfd + 12 * nab].reshape(-1, 12)
        err = max(err, np.max(np.abs(qg[:, :3] - qo[:, :3])) / S.L, np.max(np.abs(qg[:, 3:] - qo[:, 3:])))
    return err, st


GRASP_STEPS = [2, 4, 7, 10, 12, 14]   # contact onset, squeeze, squeeze, hold, lift (bases rise from step 12)


def test_grasp_fp64_matches_oracle(grasp):
    sc, S, states = grasp
    sim = _sim(sc)
    worst = 0.0
    pairs = 0
    for k in GRASP_STEPS:
        err, st = _teacher_forced_step(sim, sc, S, states, k)
        worst = max(worst, err)
        pairs = max(pairs, st["n_pairs_max"])
        assert st["n_friction_pairs"] > 0 or k < 3
    assert pairs > 20
    assert worst < 1e-8, worst


def test_grasp_mixed_precision_matches_oracle(grasp):
    from paper_2609_25653_b300 import ipcsim
    sc, S, states = grasp
    sim = _sim(sc, precision=ipcsim.PREC_MIXED, newton_tol=1e-6, pcg_rtol=1e-4)
    worst = max(_teacher_forced_step(sim, sc, S, states, k)[0] for k in GRASP_STEPS)
    assert worst < 1e-5, worst


@pytest.mark.parametrize("streamed", [False, True])
def test_grasp_every_pcg_shape_matches_oracle(grasp, streamed):
    """Each (threads per FEM row, CTAs per SM) the autotuner may pick, with the operator staged in shared
    memory or streamed from global memory in every iteration, reaches the oracle's state."""
    sc, S, states = grasp
    sim = _sim(sc)
    sim.pcg_residency(streamed)
    k = 9
    for bps in (1, 2):
        for rowg in (1, 2, 4, 8):
            sim.tuning(rowg=rowg, blocks_per_sm=bps)
            err, _ = _teacher_forced_step(sim, sc, S, states, k)
            (r, b), _ = sim.tuning()
            grid, resident = sim.pcg_layout()
            assert (r, b) == (rowg, bps)
            assert resident == (not streamed)
            assert err < 1e-8, (rowg, bps, streamed, err)


def test_grasp_mixed_streamed_operator_matches_oracle(grasp):
    from paper_2609_25653_b300 import ipcsim
    sc, S, states = grasp
    sim = _sim(sc, precision=ipcsim.PREC_MIXED, newton_tol=1e-6, pcg_rtol=1e-4)
    sim.pcg_residency(True)
    for k in (7, 12):
        err, _ = _teacher_forced_step(sim, sc, S, states, k)
        assert sim.pcg_layout()[1] is False
        assert err < 1e-5, (k, err)


CYL_STEPS = [1, 3, 6, 9, 11]


def test_soft_cylinder_fp64_matches_oracle(cylinder):
    sc, S, states = cylinder
    sim = _sim(sc)
    worst, pairs = 0.0, 0
    for k in CYL_STEPS:
        err, st = _teacher_forced_step(sim, sc, S, states, k)
        worst = max(worst, err)
        pairs = max(pairs, st["n_pairs_max"])
    assert pairs > 300
    assert worst < 1e-8, worst


def test_soft_cylinder_mixed_precision_matches_oracle(cylinder):
    from paper_2609_25653_b300 import ipcsim
    sc, S, states = cylinder
    sim = _sim(sc, precision=ipcsim.PREC_MIXED, newton_tol=1e-6, pcg_rtol=1e-4)
    worst = max(_teacher_forced_step(sim, sc, S, states, k)[0] for k in CYL_STEPS)
    assert worst < 1e-5, worst


def test_two_level_preconditioner_reaches_the_oracle_in_fewer_iterations(grasp):
    """The coarse rigid-body correction changes the PCG's iterates, not the Newton step it solves for:
    both preconditioners reach the oracle's next state, the two-level one with fewer PCG iterations."""
    from paper_2609_25653_b300 import ipcsim
    sc, S, states = grasp
    two = _sim(sc)
    jac = _sim(sc, preconditioner=ipcsim.PRECOND_BLOCK_JACOBI)
    it_two = it_jac = 0
    for k in (4, 10, 13):
        e2, s2 = _teacher_forced_step(two, sc, S, states, k)
        ej, sj = _teacher_forced_step(jac, sc, S, states, k)
        assert e2 < 1e-8 and ej < 1e-8, (k, e2, ej)
        it_two += s2["pcg_iters_total"]
        it_jac += sj["pcg_iters_total"]
    assert it_two < it_jac, (it_two, it_jac)


def test_two_level_mixed_precision_batch_matches_single_scenes():
    """Batches run one coarse level per scene (one dense block per independent solve)."""
    from paper_2609_25653_b300 import ipcsim
    scs = [scenes.arm_gripper_grasp_reduced(s, n_steps=6) for s in (0, 1)]
    batch = ipcsim.Simulator.batch(scs, precision=ipcsim.PREC_MIXED)
    single = [_sim(sc, precision=ipcsim.PREC_MIXED) for sc in scs]
    for k in range(4):
        st = batch.step()
        assert st["status"] == 0
        xb = batch.get_state()[0]
        off = 0
        for sim in single:
            sim.step()
            xs = sim.get_state()[0]
            assert np.max(np.abs(xb[off:off + sim.nf] - xs)) / sim.L < 1e-5
            off += sim.nf
