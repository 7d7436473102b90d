"""The seeded synthetic workloads (paper_2609_25653_b300/scenes.py) that the benchmark and the parity tests
use: reproducible from their seed, the sizes the benchmark reports, every rest tet positively oriented,
kinematic trajectories made of rigid transforms, and batches whose scenes keep their own rows contiguous
(the per-scene PCG needs that)."""
import numpy as np
import pytest

from paper_2609_25653_b300 import ipcsim, scenes


def _signed_volumes(X, T):
    a, b, c, d = (X[T[:, k]] for k in range(4))
    return np.einsum("ij,ij->i", np.cross(b - a, c - a), d - a) / 6.0


def _same(s1, s2):
    for k in ("fem_X", "fem_tets", "fem_logE", "kin_T"):
        assert np.array_equal(np.asarray(s1[k]), np.asarray(s2[k])), k


def test_arm_gripper_grasp_is_reproducible_and_has_the_reported_sizes():
    a, b = scenes.arm_gripper_grasp(0), scenes.arm_gripper_grasp(0)
    _same(a, b)
    assert a["fem_X"].shape == (10336, 3) and a["fem_tets"].shape == (47472, 4)
    assert len(a["abd"]) == 1 and len(a["kin"]) == 10
    assert np.all(_signed_volumes(a["fem_X"], a["fem_tets"]) > 0)


def test_soft_gripper_cylinder_sizes_and_orientation():
    c = scenes.soft_gripper_cylinder(0, n_steps=300, close_per_step=0.25e-3)
    assert c["fem_X"].shape == (22545, 3) and c["fem_tets"].shape == (110640, 4)
    assert np.all(_signed_volumes(c["fem_X"], c["fem_tets"]) > 0)


@pytest.mark.parametrize("maker", [lambda: scenes.arm_gripper_grasp(0), lambda: scenes.fingertip_press(0, n_steps=8)])
def test_kinematic_trajectories_are_rigid(maker):
    T = np.asarray(maker()["kin_T"])  # (steps, bodies, 3, 4)
    R = T[..., :3]
    eye = np.broadcast_to(np.eye(3), R.shape)
    assert np.allclose(np.einsum("...ji,...jk->...ik", R, R), eye, atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)


def test_batched_grasps_reproducible_uneven_and_contiguous():
    b1, b2 = scenes.batched_grasps(4), scenes.batched_grasps(4)
    assert len(b1) == 4
    for s1, s2 in zip(b1, b2):
        _same(s1, s2)
        assert np.all(_signed_volumes(s1["fem_X"], s1["fem_tets"]) > 0)
    sizes = [len(s["fem_tets"]) for s in b1]
    assert len(set(sizes)) > 1  # uneven mesh sizes across the batch
    view = ipcsim.batch_scene(b1)
    # the batch concatenates FEM vertices scene by scene, so every scene's rows are one contiguous range
    counts = [len(s["fem_X"]) for s in b1]
    assert len(view["fem_X"]) == sum(counts)
    off = 0
    for s in b1:
        n = len(s["fem_X"])
        assert np.array_equal(view["fem_X"][off:off + n], s["fem_X"])
        off += n
