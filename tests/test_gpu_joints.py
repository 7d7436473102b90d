"""Joint drives (E_joint of Eq. 3) on the GPU against the oracle.

The jointed arm: three affine links on revolute joints (hinge point springs plus direction drives whose
targets turn every step) sweep into a soft block on the ground.  The CUDA path starts from the oracle's
state at sampled steps (teacher forcing) and must reach the oracle's next state (1e-8 of the bounding-box
diagonal in FP64, 1e-5 in mixed precision); a batch of two arms with different joint counts must match the
arms simulated alone; the adjoint of a jointed step must match the oracle's dense adjoint."""
import numpy as np
import pytest

from oracle import ipc as orc
from paper_2609_25653_b300 import scenes
from tests.conftest import oracle_trajectory

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PARITY = dict(newton_tol=1e-9, pcg_rtol=1e-12)
STEPS = [0, 1, 2, 4, 7, 10]


@pytest.fixture(scope="module")
def arm():
    sc = scenes.jointed_arm(3, n_steps=12, **PARITY)
    S, states = oracle_trajectory(sc)
    return sc, S, states


def _sim(sc, **kw):
    from paper_2609_25653_b300 import ipcsim
    return ipcsim.Simulator(sc, **kw)


def _forced(sim, sc, S, states, k):
    nfd, nab = S.n_fem_dof, S.nab
    z, zd = states[k]
    sim.set_state(z[:nfd].reshape(-1, 3), zd[:nfd].reshape(-1, 3), z[nfd:nfd + 12 * nab].reshape(-1, 12),
                  zd[nfd:nfd + 12 * nab].reshape(-1, 12))
    sim.set_kinematic(sc["kin_T"][k])
    sim.step_index = k
    st = sim.step()
    assert st["status"] == 0 and st["min_dist"] > 0
    xg, _, qg, _ = sim.get_state()
    zn = states[k + 1][0]
    qo = zn[nfd:nfd + 12 * nab].reshape(-1, 12)
    err = max(np.max(np.abs(xg - zn[:nfd].reshape(-1, 3))) / S.L, np.max(np.abs(qg[:, :3] - qo[:, :3])) / S.L,
              np.max(np.abs(qg[:, 3:] - qo[:, 3:])))
    return err, st


def test_jointed_arm_fp64_matches_oracle(arm):
    sc, S, states = arm
    sim = _sim(sc)
    worst, pairs = 0.0, 0
    for k in STEPS:
        err, st = _forced(sim, sc, S, states, k)
        worst = max(worst, err)
        pairs = max(pairs, st["n_pairs_max"])
    assert pairs > 9  # the arm reaches the block, not only the block the ground
    assert worst < 1e-8, worst


def test_jointed_arm_mixed_precision_matches_oracle(arm):
    from paper_2609_25653_b300 import ipcsim
    sc, S, states = arm
    sim = _sim(sc, precision=ipcsim.PREC_MIXED, pcg_rtol=1e-7)
    worst = max(_forced(sim, sc, S, states, k)[0] for k in STEPS)
    assert worst < 1e-5, worst


def test_joint_drive_angles_follow_the_targets(arm):
    """After the ramp the links hold the commanded relative angles (0.6, -0.3, 0.6 rad)."""
    sc, S, _ = arm
    sim = _sim(sc)
    for _ in range(12):
        sim.step()
    _, _, q, _ = sim.get_state()
    ang = [np.arctan2(q[i, 4], q[i, 3]) for i in range(3)]
    rel = [ang[0], ang[1] - ang[0], ang[2] - ang[1]]
    assert np.allclose(rel, [0.6, -0.3, 0.6], atol=2e-3), rel


def test_jointed_arms_batch_matches_single_scenes():
    from paper_2609_25653_b300 import ipcsim
    scs = [scenes.jointed_arm(3, n_steps=6, **PARITY), scenes.jointed_arm(2, n_steps=6, swing=-0.4, **PARITY)]
    singles = [_sim(s) for s in scs]
    batch = ipcsim.Simulator.batch(scs)
    assert batch.nj == sum(len(s["joints"]) for s in scs)
    for _ in range(6):
        for s in singles:
            assert s.step()["status"] == 0
        assert batch.step()["status"] == 0
    xb, _, qb, _ = batch.get_state()
    off_x, off_q = 0, 0
    for s, sc in zip(singles, scs):
        x, _, q, _ = s.get_state()
        L = orc.Scene(sc).L
        assert np.max(np.abs(xb[off_x:off_x + len(x)] - x)) < 1e-7 * L
        assert np.max(np.abs(qb[off_q:off_q + len(q)] - q)) < 1e-7
        off_x += len(x)
        off_q += len(q)


def test_jointed_step_adjoint_matches_oracle_dense():
    sc = scenes.jointed_arm(3, n_steps=3, newton_tol=1e-10, pcg_rtol=1e-13, max_newton=300)
    o = orc.Oracle(sc)
    o.step()
    S = o.S
    z_t, zd_t = S.z0.copy(), S.zd0.copy()
    r = np.random.default_rng(5)
    nF = S.n_free
    gz = np.zeros(S.ndof); gz[:nF] = r.normal(size=nF)
    gzd = np.zeros(S.ndof); gzd[:nF] = 1e-2 * r.normal(size=nF)
    gz_t, gzd_t, dlogE, dmu = orc.adjoint_step(o, z_t, zd_t, o.z, 1, gz, gzd)
    sim = _sim(sc)

    def dev(a):
        return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")

    T = sc["kin_T"]
    g_z, g_zd, g_logE, g_mu = sim.adjoint(dev(z_t[:nF]), dev(zd_t[:nF]), dev(o.z[:nF]), T[0], T[1], dev(gz[:nF]),
                                          dev(gzd[:nF]), step_next=1)

    def rel(a, b):
        return np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel(g_z.cpu().numpy(), gz_t[:nF]) < 1e-6
    assert rel(g_zd.cpu().numpy(), gzd_t[:nF]) < 1e-6
    assert rel(g_logE.cpu().numpy(), dlogE) < 1e-6
