"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the
same seeded inputs: per-tet elasticity, active contact sets (bit-exact),
barrier energy/gradient/Hessian, CCD step bounds, and whole steps."""
import math

import numpy as np
import pytest

from oracle import ipc as orc
from paper_2609_25653_b300 import scenes

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _sim(sc, **kw):
    from paper_2609_25653_b300 import ipcsim
    return ipcsim.Simulator(sc, **kw)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def all_positions(S, sim, xf):
    """Global vertex array (FEM | ABD | kinematic) for FEM positions xf and the scene's initial poses."""
    z = S.z0.copy()
    z[:S.n_fem_dof] = xf.reshape(-1)
    return S.positions(z)


def canon(rec, s):
    """Set of (kind, type, v0..v3) -> s; independent of primitive numbering."""
    out = {}
    for r, sv in zip(rec, s):
        out[(int(r[0]), int(r[3]), int(r[4]), int(r[5]), int(r[6]), int(r[7]))] = float(sv)
    return out


def deformed_press_positions(seed):
    sc = scenes.fingertip_press(seed)
    S = orc.Scene(sc)
    r = np.random.default_rng(seed)
    X = sc["fem_X"].copy()
    # squash towards the cube and the plate, with a random smooth field
    X[:, 2] = 0.5e-3 + (X[:, 2] - 0.5e-3) * 0.96 - 0.35e-3
    X += 5e-5 * r.normal(size=X.shape)
    return sc, S, X


def test_elastic_parity():
    sc, S, X = deformed_press_positions(1)
    sim = _sim(sc)
    for project in (False, True):
        E, g, H = sim.eval_elastic(_dev(X), project=project)
        Eo = np.zeros(1)
        go = np.zeros(3 * S.nf)
        Ho = np.zeros(len(S.tets) * 144)
        import ctypes as C
        Ec = C.c_double(0.0)
        orc.lib().orc_elastic_all(len(S.tets), orc._i(S.tets), orc._d(S.B), orc._d(S.vol), orc._d(S.mu),
                                  orc._d(S.lam), orc._d(np.ascontiguousarray(X.reshape(-1))), int(project),
                                  C.byref(Ec), orc._d(go), orc._d(Ho))
        assert abs(E.item() - Ec.value) <= 1e-12 * abs(Ec.value)
        gg = g.cpu().numpy().reshape(-1)
        assert np.max(np.abs(gg - go)) <= 1e-11 * np.max(np.abs(go))
        HH = H.cpu().numpy().reshape(-1)
        assert np.max(np.abs(HH - Ho)) <= 1e-9 * np.max(np.abs(Ho))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_active_set_bit_exact(seed):
    sc, S, X = deformed_press_positions(seed)
    sim = _sim(sc)
    xv = all_positions(S, sim, X)
    # move the plate down onto the box as well
    xv[S.nf + S.na_v + 8:] += np.array([0, 0, -0.45e-3])
    rec_g, s_g = sim.active_pairs(_dev(xv))
    rec_o, s_o = S.active_pairs(np.ascontiguousarray(xv.reshape(-1)))
    A = canon(rec_g.cpu().numpy(), s_g.cpu().numpy())
    B = canon(rec_o, s_o)
    assert len(B) > 20
    assert set(A) == set(B)
    for k in B:
        assert A[k] == B[k]  # bit-exact squared distances


def test_barrier_parity():
    sc, S, X = deformed_press_positions(0)
    sim = _sim(sc)
    xv = all_positions(S, sim, X)
    xv[S.nf + S.na_v + 8:] += np.array([0, 0, -0.45e-3])
    rec_g, s_g = sim.active_pairs(_dev(xv))
    assert rec_g.shape[0] > 0
    for project in (False, True):
        E, g, H = sim.eval_barrier(_dev(xv), rec_g, project=project)
        rec = rec_g.cpu().numpy()
        Ho = []
        Eo = 0.0
        go = np.zeros((S.nv, 3))
        epsx = S.eps_x(rec)
        for k in range(len(rec)):
            ids = rec[k, 4:8]
            e, gk, hk = orc.pair(int(rec[k, 0]), int(rec[k, 3]), xv[ids], S.sh, S.kappa, epsx[k], project)
            Eo += e
            np.add.at(go, ids, gk.reshape(4, 3))
            Ho.append(hk)
        assert abs(E.item() - Eo) <= 1e-12 * abs(Eo)
        gF = g.cpu().numpy()[:S.nf]
        assert np.max(np.abs(gF - go[:S.nf])) <= 1e-10 * np.max(np.abs(go[:S.nf]))
        Hg = H.cpu().numpy()
        for k in range(len(rec)):
            scale = max(np.max(np.abs(Ho[k])), 1e-300)
            assert np.max(np.abs(Hg[k] - Ho[k])) <= 1e-8 * scale


def test_ccd_parity():
    sc, S, X = deformed_press_positions(2)
    sim = _sim(sc)
    xv = all_positions(S, sim, X)
    r = np.random.default_rng(5)
    for trial in range(3):
        p = np.zeros_like(xv)
        p[:S.nf] = 1e-3 * r.normal(size=(S.nf, 3)) + np.array([0, 0, -1.5e-3])
        p[S.nf + S.na_v + 8:] = np.array([0, 0, -1.2e-3])
        a_g, n_g = sim.ccd_alpha(_dev(xv), _dev(p))
        a_o, n_o = _oracle_ccd(S, xv, p)
        assert n_g == n_o
        assert a_g == a_o
        assert 0 < a_g < 1


def _oracle_ccd(S, xv, p):
    import ctypes as C
    nc = C.c_int()
    a = orc.lib().orc_ccd_alpha(C.byref(S.surf), orc._d(np.ascontiguousarray(xv.reshape(-1))),
                                orc._d(np.ascontiguousarray(p.reshape(-1))), S.s_ccd, orc.ACCD_MAX_ITER, C.byref(nc))
    return a, nc.value


def test_free_fall_exact():
    sc = scenes.free_block(n_steps=4, v0=(0.1, -0.2, 0.3))
    sim = _sim(sc, newton_tol=1e-12, pcg_rtol=1e-14)
    x = sc["fem_X"].copy()
    v = np.array([0.1, -0.2, 0.3])
    dt = sc["params"]["dt"]
    for _ in range(4):
        st = sim.step()
        v = v + dt * sc["gravity"]
        x = x + dt * v
        xg, vg, _, _ = sim.get_state()
        # closed form up to the PCG's residual (relative 1e-14 of a 4 mm displacement)
        assert np.max(np.abs(xg - x)) < 1e-13
        assert np.max(np.abs(vg - v)) < 1e-10


PARITY = dict(newton_tol=1e-9, pcg_rtol=1e-12)


def test_step_parity_teacher_forced():
    """Both sides start every step from the oracle's state; positions agree to 1e-8 of the bbox diagonal."""
    sc = scenes.fingertip_press(0, n_steps=6, **PARITY)
    o = orc.Oracle(sc)
    sim = _sim(sc)
    worst = 0.0
    for k in range(6):
        x0 = o.x()[:o.S.nf].copy()
        v0 = o.zd[:o.S.n_fem_dof].reshape(-1, 3).copy()
        sim.set_state(x0, v0)
        st = sim.step()
        o.step()
        xg, _, _, _ = sim.get_state()
        err = np.max(np.abs(xg - o.x()[:o.S.nf])) / o.S.L
        worst = max(worst, err)
        assert st["status"] == 0 and st["min_dist"] > 0
    assert worst < 1e-8, worst


def test_trajectory_parity_20_steps():
    sc = scenes.fingertip_press(0, n_steps=20, **PARITY)
    o = orc.Oracle(sc)
    sim = _sim(sc)
    errs = []
    for k in range(20):
        sim.step()
        o.step()
        xg, vg, _, _ = sim.get_state()
        errs.append(np.max(np.abs(xg - o.x()[:o.S.nf])) / o.S.L)
    assert max(errs) < 1e-8, errs


def test_newton_cap_restores_state():
    sc = scenes.fingertip_press(0, n_steps=2)
    sim = _sim(sc, max_newton=1)
    x0, v0, _, _ = sim.get_state()
    st = sim.step(raise_on_error=False)
    assert st["status"] == -4
    x1, v1, _, _ = sim.get_state()
    assert np.array_equal(x0, x1) and np.array_equal(v0, v1)


def test_inverted_tet_rejected():
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.free_block()
    sc["fem_tets"] = sc["fem_tets"].copy()
    sc["fem_tets"][0, [1, 2]] = sc["fem_tets"][0, [2, 1]]
    with pytest.raises(ipcsim.IpcError) as e:
        _sim(sc)
    assert e.value.code == -2


def test_initial_intersection_rejected():
    """A vertex lying exactly on a kinematic triangle (distance 0) is refused at create."""
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.free_block(n_steps=2)
    mm = 1e-3
    gX = np.array([[-10 * mm, -10 * mm, 0.0], [20 * mm, -10 * mm, 0.0], [-10 * mm, 20 * mm, 0.0]])
    sc["kin"] = [dict(X=gX, tris=np.array([[0, 1, 2]], np.int32))]
    sc["kin_T"] = np.tile(scenes.translation((0, 0, 0)), (3, 1, 1, 1))
    with pytest.raises(ipcsim.IpcError) as e:
        _sim(sc)
    assert e.value.code == -3


@pytest.mark.parametrize("name", ["abd_box_drop", "stitched_block"])
def test_abd_and_stitch_parity(name):
    """Affine-body contact and stitch springs: teacher-forced steps agree with the oracle to 1e-8 L."""
    sc = getattr(scenes, name)(n_steps=6, **PARITY)
    o = orc.Oracle(sc)
    sim = _sim(sc)
    nfd, nab = o.S.n_fem_dof, o.S.nab
    for k in range(6):
        x0 = o.z[:nfd].reshape(-1, 3).copy()
        v0 = o.zd[:nfd].reshape(-1, 3).copy()
        q0 = o.z[nfd:nfd + 12 * nab].reshape(-1, 12).copy() if nab else None
        qd0 = o.zd[nfd:nfd + 12 * nab].reshape(-1, 12).copy() if nab else None
        sim.set_state(x0, v0, q0, qd0)
        st = sim.step()
        o.step()
        xg, _, qg, _ = sim.get_state()
        err = np.max(np.abs(xg - o.z[:nfd].reshape(-1, 3))) / o.S.L
        assert err < 1e-8, (k, err)
        if nab:
            qo = o.z[nfd:nfd + 12 * nab].reshape(-1, 12)
            assert np.max(np.abs(qg[:, :3] - qo[:, :3])) / o.S.L < 1e-8
            assert np.max(np.abs(qg[:, 3:] - qo[:, 3:])) < 1e-8


def test_lbvh_matches_all_pairs_on_grasp_scene():
    """The LBVH broad phase returns exactly the all-pairs active set on the arm-gripper geometry."""
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.arm_gripper_grasp(0, n_steps=4)
    a = _sim(sc)
    b = _sim(sc, broad_phase=ipcsim.BROAD_ALL_PAIRS)
    S = orc.Scene(sc)
    xv = S.positions(S.z0).copy()
    # squeeze the fingertips onto the object so that many pairs are active
    r = np.random.default_rng(0)
    xv[:S.nf, 1] *= 0.985
    xv[:S.nf] += 2e-5 * r.normal(size=(S.nf, 3))
    ra, sa = a.active_pairs(_dev(xv))
    rb, sb = b.active_pairs(_dev(xv))
    A = canon(ra.cpu().numpy(), sa.cpu().numpy())
    B = canon(rb.cpu().numpy(), sb.cpu().numpy())
    assert len(B) > 50 and A == B
    p = np.zeros_like(xv)
    p[:S.nf, 1] = -1e-3 * np.sign(xv[:S.nf, 1])
    p[:S.nf] += 1e-4 * r.normal(size=(S.nf, 3))
    assert a.ccd_alpha(_dev(xv), _dev(p)) == b.ccd_alpha(_dev(xv), _dev(p))


def test_mixed_precision_within_1e5():
    """FP32 operator / FP64 residual path: positions within 1e-5 of the bbox diagonal of the FP64 path and the oracle."""
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.fingertip_press(0, n_steps=8)
    a = _sim(sc)
    b = _sim(sc, precision=ipcsim.PREC_MIXED)
    o = orc.Oracle(sc)
    for k in range(8):
        sa = a.step()
        sb = b.step()
        o.step()
        xa = a.get_state()[0]
        xb = b.get_state()[0]
        L = o.S.L
        assert np.max(np.abs(xa - xb)) / L < 1e-5
        assert np.max(np.abs(xb - o.x()[:o.S.nf])) / L < 1e-5
        assert sb["status"] == 0 and sb["min_dist"] > 0


def test_step_many_matches_single_scene_steps():
    """Concurrent stepping of independent scenes (one stream and host thread each) gives each scene's own result."""
    from paper_2609_25653_b300 import ipcsim
    scs = [scenes.fingertip_press(s, n_steps=4, **PARITY) for s in (0, 1, 2)] + [scenes.abd_box_drop(n_steps=4, **PARITY)]
    streams = [torch.cuda.Stream() for _ in scs]
    many = [_sim(sc, stream=st) for sc, st in zip(scs, streams)]
    single = [_sim(sc) for sc in scs]
    for k in range(4):
        stats = ipcsim.step_many(many)
        assert all(s["status"] == 0 for s in stats)
        for sim in single:
            sim.step()
        for a, b in zip(many, single):
            xa, _, qa, _ = a.get_state()
            xb, _, qb, _ = b.get_state()
            assert np.max(np.abs(xa - xb)) <= 1e-9 * b.L
            if a.nab:
                assert np.max(np.abs(qa - qb)) <= 1e-9


def test_batch_matches_individual_scenes():
    """Independent scenes concatenated into one simulator give each scene's own trajectory."""
    from paper_2609_25653_b300 import ipcsim
    scs = [scenes.fingertip_press(s, n_steps=4, **PARITY) for s in (0, 1, 2)]
    batch = ipcsim.Simulator.batch(scs)
    single = [_sim(sc) for sc in scs]
    assert batch.n_scenes == 3 and batch.nf == sum(s.nf for s in single)
    for k in range(4):
        st = batch.step()
        assert st["status"] == 0 and st["min_dist"] > 0
        xb = batch.get_state()[0]
        off = 0
        for sim in single:
            sim.step()
            xs = sim.get_state()[0]
            assert np.max(np.abs(xb[off:off + sim.nf] - xs)) <= 1e-8 * sim.L
            off += sim.nf


def test_batch_scenes_keep_their_own_newton_path():
    """Scenes of a batch that need different step lengths (one plate presses three times faster) keep
    their own convergence test, CCD bound and line search: each matches its own simulation."""
    from paper_2609_25653_b300 import ipcsim
    a = scenes.fingertip_press(0, n_steps=6, **PARITY)
    b = scenes.fingertip_press(1, n_steps=6, **PARITY)
    kin_T = b["kin_T"].copy()
    for s in range(kin_T.shape[0]):
        kin_T[s, 1, 2, 3] = 21e-3 - 0.3e-3 * s
    b["kin_T"] = kin_T
    batch = ipcsim.Simulator.batch([a, b])
    single = [_sim(a), _sim(b)]
    for k in range(6):
        st = batch.step()
        assert st["status"] == 0 and st["min_dist"] > 0
        xb = batch.get_state()[0]
        off = 0
        for sim in single:
            sim.step()
            xs = sim.get_state()[0]
            assert np.max(np.abs(xb[off:off + sim.nf] - xs)) <= 1e-8 * sim.L
            off += sim.nf


def test_batch_mixed_scenes_within_1e5():
    """Mixed precision on a batch whose scenes converge at different Newton and PCG iterations (each scene
    has its own FP32 solve, refinement and stop; converged scenes are left out): every scene stays within
    1e-5 of the bbox diagonal of its own FP64 simulation."""
    from paper_2609_25653_b300 import ipcsim
    a = scenes.fingertip_press(0, n_steps=6)
    b = scenes.fingertip_press(1, n_steps=6)
    kin_T = b["kin_T"].copy()
    for s in range(kin_T.shape[0]):
        kin_T[s, 1, 2, 3] = 21e-3 - 0.3e-3 * s
    b["kin_T"] = kin_T
    batch = ipcsim.Simulator.batch([a, b], precision=ipcsim.PREC_MIXED)
    single = [_sim(a), _sim(b)]
    for k in range(6):
        st = batch.step()
        assert st["status"] == 0 and st["min_dist"] > 0
        xb = batch.get_state()[0]
        off = 0
        for sim in single:
            sim.step()
            xs = sim.get_state()[0]
            assert np.max(np.abs(xb[off:off + sim.nf] - xs)) / sim.L < 1e-5
            off += sim.nf


@pytest.mark.parametrize("name", ["fingertip_press", "abd_box_drop"])
def test_sweep_candidates_match_all_pairs_steps(name):
    """Whole steps with the LBVH sweep (candidates filtered along the line search) equal all-pairs culling."""
    from paper_2609_25653_b300 import ipcsim
    sc = getattr(scenes, name)(n_steps=5, **PARITY) if name != "fingertip_press" else scenes.fingertip_press(0, n_steps=5, **PARITY)
    a = _sim(sc)
    b = _sim(sc, broad_phase=ipcsim.BROAD_ALL_PAIRS)
    for k in range(5):
        sa = a.step()
        sb = b.step()
        assert sa["status"] == 0 and sb["status"] == 0
        xa, _, qa, _ = a.get_state()
        xb, _, qb, _ = b.get_state()
        assert np.max(np.abs(xa - xb)) <= 1e-8 * a.L


def test_soft_cylinder_mixed_within_1e5():
    """Two fingertips squeezing a deformable cylinder (about 110k tets in all): the FP32-iteration path
    stays within 1e-5 of the bbox diagonal of the FP64 path while contact builds up."""
    from paper_2609_25653_b300 import ipcsim
    sc = scenes.soft_gripper_cylinder(0, n_steps=8, close_per_step=0.25e-3)
    a = _sim(sc)
    b = _sim(sc, precision=ipcsim.PREC_MIXED)
    for k in range(8):
        sa = a.step()
        sb = b.step()
        assert sa["status"] == 0 and sb["status"] == 0
        xa = a.get_state()[0]
        xb = b.get_state()[0]
        assert np.max(np.abs(xa - xb)) / a.L < 1e-5
    assert sa["n_pairs_max"] > 0 and sa["min_dist"] > 0 and sb["min_dist"] > 0
