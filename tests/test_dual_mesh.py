"""Physics-to-render dual-mesh mapping (§III-D.1, Eqs. 5-6).

CPU: the oracle's Loop subdivision against hand-derived values and invariants, and the library's
host-built W against the oracle's.  GPU: X_f = W X_c on the device against the oracle's sparse product."""
import math

import numpy as np
import pytest

from oracle import dual_mesh as dm
from oracle import ipc as orc
from paper_2609_25653_b300 import scenes

TET_X = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
TET_T = np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]])


def test_loop_tetrahedron_by_hand():
    """One level on a tetrahedron: every vertex has valence 3, beta(3) = (5/8 - (3/8 - 1/8)^2) / 3 = 3/16, so
    an old vertex moves to 7/16 v + 3/16 (sum of the other three); the edge (0, 1) has opposite vertices 2
    and 3, so its new vertex is 3/8 (x0 + x1) + 1/8 (x2 + x3)."""
    assert dm.loop_beta(3) == pytest.approx(3.0 / 16.0, abs=1e-15)
    W, t = dm.subdivision_matrix(TET_T, 4, 1)
    Wd = W.toarray()
    for v in range(4):
        for u in range(4):
            assert Wd[v, u] == pytest.approx(7.0 / 16.0 if u == v else 3.0 / 16.0, abs=1e-15)
    # edges in sorted order: (0,1) (0,2) (0,3) (1,2) (1,3) (2,3) -> vertices 4..9
    assert np.allclose(Wd[4], [0.375, 0.375, 0.125, 0.125])
    assert np.allclose(Wd[9], [0.125, 0.125, 0.375, 0.375])
    assert t.shape == (16, 3)


@pytest.mark.parametrize("levels", [1, 2, 3])
def test_loop_counts_affine_invariance_and_orientation(levels):
    """V' = V + E, F' = 4 F per level (a closed mesh keeps V - E + F = 2); rows of W sum to one (an affine
    map of the coarse mesh maps the fine mesh the same way); triangles keep their outward orientation."""
    W, t = dm.subdivision_matrix(TET_T, 4, levels)
    V, F = 4, 4
    E = 6
    for _ in range(levels):
        V, E, F = V + E, 2 * E + 3 * F, 4 * F
    assert W.shape == (V, 4) and len(t) == F and V - E + F == 2
    assert np.allclose(np.asarray(W.sum(1)).ravel(), 1.0, atol=1e-14)
    A = np.array([[1.3, 0.2, -0.4], [0.1, 0.7, 0.5], [-0.3, 0.2, 1.1]])
    b = np.array([0.3, -1.0, 2.0])
    Xf = dm.fine_positions(W, TET_X)
    assert np.allclose(dm.fine_positions(W, TET_X @ A.T + b), Xf @ A.T + b, atol=1e-13)
    # signed volume of the closed fine surface stays positive (outward triangles)
    a, bb, c = Xf[t[:, 0]], Xf[t[:, 1]], Xf[t[:, 2]]
    assert np.einsum("ij,ij->i", a, np.cross(bb, c)).sum() > 0


def test_loop_planar_patch_stays_planar():
    """Subdivision of a planar patch stays in its plane (the rules are affine combinations)."""
    X, T = scenes.grid_tets((0.0, 0.0, 0.0), 1.0, 3, 3, 1)
    S = orc.extract_surface(T)
    W, t = dm.subdivision_matrix(S, len(X), 2)
    Xf = dm.fine_positions(W, X)
    used = np.unique(t)
    top = [v for v in used if W[v].nnz and np.all(np.abs(X[W[v].indices, 2] - 1.0) < 1e-12)]
    assert len(top) > 10
    assert np.allclose(Xf[top, 2], 1.0, atol=1e-14)


def _tip_surface():
    sc = scenes.arm_gripper_grasp_reduced(0, n_steps=1)
    T = sc["fem_tets"]
    fb = sc["fem_body"]
    return sc["fem_X"], orc.extract_surface(T[fb == 0])


@pytest.mark.parametrize("levels", [1, 2])
def test_library_matrix_equals_oracle(levels):
    """The library's host-built W (sim_dual_mesh_topology, no GPU) equals the oracle's, entry by entry."""
    from paper_2609_25653_b300 import ipcsim
    X, S = _tip_surface()
    Wo, to = dm.subdivision_matrix(S, len(X), levels)
    m = ipcsim.DualMesh(S, len(X), levels, upload=False)
    tl, Wl = m.topology()
    assert Wl.shape == Wo.shape and Wl.nnz == Wo.nnz
    assert np.array_equal(Wl.indptr, Wo.indptr) and np.array_equal(Wl.indices, Wo.indices)
    assert np.max(np.abs(Wl.data - Wo.data)) <= 1e-15
    assert np.array_equal(np.sort(np.sort(tl, 1), 0), np.sort(np.sort(to, 1), 0))


@pytest.mark.gpu
def test_gpu_fine_positions_match_oracle():
    torch = pytest.importorskip("torch")
    from paper_2609_25653_b300 import ipcsim
    X, S = _tip_surface()
    r = np.random.default_rng(2)
    Xc = X + 1e-4 * r.normal(size=X.shape)
    W, _ = dm.subdivision_matrix(S, len(X), 3)
    m = ipcsim.DualMesh(S, len(X), 3)
    xf = m.apply(torch.as_tensor(Xc, device="cuda"))
    torch.cuda.synchronize()
    ref = dm.fine_positions(W, Xc)
    assert np.max(np.abs(xf.cpu().numpy() - ref)) <= 1e-15 * np.max(np.abs(ref)) * 8
