"""Host logic of the cooperative PCG: how the rows of the Newton system are split among the CTAs
(sim_pcg_partition, no GPU).  A batch of scenes gets one independent solve per scene only if every CTA's
rows lie in one scene; the rows are covered exactly once; the FEM rows are balanced by stored blocks."""
import numpy as np
import pytest

from paper_2609_25653_b300 import ipcsim


def _system(rng, scene_fem, scene_abd):
    """BSR row offsets and the scene of every row for scenes with the given FEM vertex and ABD body counts."""
    nf, nab = int(sum(scene_fem)), int(sum(scene_abd))
    node_scene = np.concatenate([np.repeat(np.arange(len(scene_fem)), scene_fem),
                                 np.repeat(np.arange(len(scene_abd)), 4 * np.asarray(scene_abd))]).astype(np.int32)
    blocks = rng.integers(5, 25, size=nf + 4 * nab)
    row = np.concatenate([[0], np.cumsum(blocks)]).astype(np.int32)
    return row, nf, nab, node_scene


def _check(P, row, nf, nab, grid, node_scene, n_scenes):
    nfc, nac = P["n_fem_ctas"], P["n_abd_ctas"]
    seg, aseg, cs = P["seg"], P["abd_seg"], P["cta_scene"]
    assert nfc >= 1 and nfc + nac <= grid
    assert (nac >= 1) == (nab > 0)
    # every row and body exactly once, in order
    assert seg[0] == 0 and seg[-1] == nf and np.all(np.diff(seg) >= 0)
    if nac:
        assert aseg[0] == 0 and aseg[-1] == nab and np.all(np.diff(aseg) >= 0)
    assert P["max_rows"] == int(np.max(np.diff(seg)))
    if P["n_solves"] == 1:
        assert np.all(cs[:nfc + nac] == 0)
        return
    assert P["n_solves"] == n_scenes
    for c in range(nfc):  # a FEM CTA serves one scene, and every row it holds belongs to it
        rows = node_scene[seg[c]:seg[c + 1]]
        if len(rows):
            assert np.all(rows == cs[c])
    for k in range(nac):
        bodies = node_scene[nf + 4 * np.arange(aseg[k], aseg[k + 1])]
        if len(bodies):
            assert np.all(bodies == cs[nfc + k])
    for s in range(n_scenes):  # every scene with rows has CTAs of its own
        if np.any(node_scene == s):
            assert np.any(cs == s)


def test_single_scene_is_one_balanced_solve():
    rng = np.random.default_rng(0)
    row, nf, nab, _ = _system(rng, [10336], [1])
    P = ipcsim.pcg_partition(row, nf, nab, 296)
    _check(P, row, nf, nab, 296, None, 1)
    assert P["n_solves"] == 1 and P["n_abd_ctas"] == 1
    seg = P["seg"]
    cost = (row[seg[1:]] - row[seg[:-1]]) + 2 * np.diff(seg)
    assert cost.max() <= 1.1 * cost.mean() + 40  # a CTA holds at most one row's cost above its share


@pytest.mark.parametrize("seed", range(40))
def test_batches_get_one_solve_per_scene(seed):
    rng = np.random.default_rng(seed)
    n_scenes = int(rng.integers(2, 40))
    fem = rng.integers(0, 400, size=n_scenes)
    fem[rng.integers(0, n_scenes)] += 1  # at least one FEM row
    abd = rng.integers(0, 3, size=n_scenes)
    grid = int(rng.integers(2, 600))
    row, nf, nab, node_scene = _system(rng, fem, abd)
    P = ipcsim.pcg_partition(row, nf, nab, grid, node_scene, n_scenes)
    _check(P, row, nf, nab, grid, node_scene, n_scenes)
    if grid >= 2 * n_scenes + 1:  # room for a FEM and an ABD CTA per scene: one solve per scene
        assert P["n_solves"] == n_scenes


def test_too_few_ctas_or_unordered_rows_fall_back_to_one_solve():
    rng = np.random.default_rng(1)
    row, nf, nab, node_scene = _system(rng, [50] * 30, [0] * 30)
    P = ipcsim.pcg_partition(row, nf, nab, 20, node_scene, 30)  # 20 CTAs for 30 scenes
    _check(P, row, nf, nab, 20, node_scene, 30)
    assert P["n_solves"] == 1
    shuffled = node_scene.copy()
    shuffled[:nf] = shuffled[:nf][::-1]  # scenes not contiguous in row order
    P = ipcsim.pcg_partition(row, nf, nab, 296, shuffled, 30)
    assert P["n_solves"] == 1
    too_many = np.repeat(np.arange(300), 2).astype(np.int32)  # more scenes than decision threads
    row2 = np.arange(0, 5 * 600 + 1, 5, dtype=np.int32)
    P = ipcsim.pcg_partition(row2, 600, 0, 900, too_many, 300)
    assert P["n_solves"] == 1


def test_contact_work_moves_rows_off_the_contact_ctas():
    """Rows with contact incidences cost more: the CTAs that own them get fewer rows, and the largest
    weighted cost of a CTA stays within one row of its share."""
    rng = np.random.default_rng(3)
    row, nf, nab, _ = _system(rng, [10000], [1])
    extra = np.zeros(nf, np.int32)
    extra[4000:4600] = 4 * rng.integers(1, 40, size=600)  # a contact patch
    plain = ipcsim.pcg_partition(row, nf, nab, 296)
    P = ipcsim.pcg_partition(row, nf, nab, 296, row_extra=extra)
    _check(P, row, nf, nab, 296, None, 1)
    pre = np.concatenate([[0], np.cumsum(np.diff(row[:nf + 1]) + 2 + extra)])
    def worst(seg):
        return int(np.max(pre[seg[1:]] - pre[seg[:-1]]))
    assert worst(P["seg"]) < worst(plain["seg"]) / 3
    per_row_max = int(np.max(np.diff(row[:nf + 1]) + 2 + extra))
    assert worst(P["seg"]) <= pre[-1] / P["n_fem_ctas"] + per_row_max


def test_partition_rejects_bad_arguments():
    row = np.arange(0, 11, dtype=np.int32)
    with pytest.raises(ValueError):
        ipcsim.pcg_partition(row, 10, 0, 1)
    with pytest.raises(ValueError):
        ipcsim.pcg_partition(row, 10, 0, 8, None, 3)
