"""Adaptive barrier stiffness on the GPU against the oracle.

The resting-cube scene of the oracle pins (a 10 mm affine cube on a ground triangle, initial kappa low
enough that its corners sink below 1e-2 dhat), with a light one-cell FEM cube resting far away so that the
scene has deformable nodes: the GPU must double kappa at the same Newton iterations as the oracle (the
per-step kappa after every step equal) and reach the oracle's positions."""
import numpy as np
import pytest

from oracle import ipc as orc
from paper_2609_25653_b300 import scenes
from tests.test_oracle_pins_kappa import DHAT, KAPPA0, _scene, rest_height

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _with_fem(sc):
    X, tets = scenes.grid_tets((0.1, 0.0, 0.5e-3), 4e-3, 1, 1, 1)
    sc = dict(sc)
    sc.update(fem_X=X, fem_tets=tets, fem_logE=np.full(len(tets), np.log(1e5)), fem_nu=np.full(len(tets), 0.3),
              fem_rho=np.full(len(tets), 1.0), fem_body=np.zeros(len(tets), np.int32))
    return sc


@pytest.mark.parametrize("adaptive", [False, True])
def test_kappa_sequence_and_rest_state_match_the_oracle(adaptive):
    from paper_2609_25653_b300 import ipcsim
    sc = _with_fem(_scene(adaptive, n_steps=20))
    o = orc.Oracle(sc)
    sim = ipcsim.Simulator(sc)
    for _ in range(20):
        o.step()
        st = sim.step()
        assert st["status"] == 0
        assert st["kappa_end"] == o.S.kappa
    x, _, q, _ = sim.get_state()
    S = o.S
    assert np.abs(x - o.z[:S.n_fem_dof].reshape(-1, 3)).max() < 1e-9 * S.L
    qo = o.z[S.n_fem_dof:S.n_fem_dof + 12]
    assert np.abs(q[0, :3] - qo[:3]).max() < 1e-9 * S.L
    assert np.abs(q[0, 3:] - qo[3:]).max() < 1e-9
    d = sim.positions().cpu().numpy()[S.nf:S.nf + 8, 2].min()
    kappa = o.S.kappa
    assert abs(d - rest_height(kappa)) <= 1e-6 * d
    assert (kappa > KAPPA0) == adaptive and (d >= 1e-2 * DHAT) == adaptive
