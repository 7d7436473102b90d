"""Pins of the oracle's joint drive potentials (E_joint of Eq. 3) against closed forms and invariants.

Each scene is a few affine boxes with joints and no contact, so the step's minimiser is fixed by the joint
springs, gravity and the affine orthogonality energy alone:
  - a box hung from a world point by one spring settles at the static sag m g / k below the anchor;
  - a box on a world hinge turns until its drive direction reaches the target angle;
  - a prismatic drive between two boxes places one at the slide offset along the other's axis;
  - joint forces between free bodies are internal: total linear momentum stays zero.
"""
import math

import numpy as np
import pytest

from oracle import ipc
from paper_2609_25653_b300 import scenes

MM = 1e-3


def _box(half, rho=1000.0, centre=(0.0, 0.0, 0.0), A=None):
    h = np.asarray(half, float)
    X, T = scenes.subdivided_box(-h, h, 1)
    A = np.eye(3) if A is None else np.asarray(A, float)
    q0 = np.concatenate([np.asarray(centre, float), A[:, 0], A[:, 1], A[:, 2]])
    return dict(X=X, tris=T, rho=rho, q0=q0)


def _scene(abd, joints, n_steps, gravity=0.0, joint_b=None, joint_t=None, **kw):
    p = scenes.default_params(dt=1e-2, dhat=0.2 * MM, mu=0.0, n_steps=n_steps, newton_tol=1e-10, pcg_rtol=1e-12,
                              max_newton=200)
    p.update(kw)
    sc = dict(name="joint_pin", fem_X=np.zeros((0, 3)), fem_tets=np.zeros((0, 4), np.int32),
              fem_logE=np.zeros(0), fem_nu=np.zeros(0), fem_rho=np.zeros(0), fem_body=np.zeros(0, np.int32),
              kin=[], kin_T=np.zeros((n_steps + 1, 0, 3, 4)), abd=abd,
              stitch_v=np.zeros(0, np.int32), stitch_b=np.zeros(0, np.int32), stitch_X=np.zeros((0, 3)),
              joints=joints, gravity=np.array([0.0, 0.0, -gravity]), params=p)
    if joint_b is not None:
        sc["joint_b"] = joint_b
    if joint_t is not None:
        sc["joint_t"] = joint_t
    return sc


def _run(sc):
    o = ipc.Oracle(sc)
    for _ in range(sc["params"]["n_steps"]):
        o.step()
    return o


def _q(o, i):
    S = o.S
    return o.z[S.n_fem_dof + 12 * i:S.n_fem_dof + 12 * (i + 1)], o.zd[S.n_fem_dof + 12 * i:S.n_fem_dof + 12 * (i + 1)]


def test_hanging_point_spring_settles_at_static_sag():
    # a 10 mm cube (1 g) hung by its top-face centre v from a world anchor.  At rest the spring carries the
    # weight, r_z = -m g / k, and the affine body stretches along z by the eps that balances the load's
    # virtual work m g v_z against the orthogonality energy kappa_A V ((1 + eps)^2 - 1)^2:
    # 4 kappa_A V (2 eps + eps^2)(1 + eps) = m g v_z; p = anchor - (1 + eps) v - (m g / k) e_z
    k, g = 10.0, 9.81
    m = 1000.0 * (10 * MM) ** 3
    kV = 1e8 * (10 * MM) ** 3
    v = (0.0, 0.0, 5 * MM)
    anchor = np.array([0.01, -0.02, 0.1])
    j = dict(a=0, a_kind=0, a_vec=v, b=-1, b_kind=0, b_vec=(0, 0, 0), k=k, t=tuple(anchor))
    sc = _scene([_box((5 * MM,) * 3, centre=anchor - np.array(v))], [j], n_steps=80, gravity=g)
    o = _run(sc)
    q, qd = _q(o, 0)
    eps = 0.0
    for _ in range(50):
        f = 4 * kV * (2 * eps + eps ** 2) * (1 + eps) - m * g * v[2]
        eps -= f / (4 * kV * (2 + 6 * eps + 3 * eps ** 2))
    assert eps > 1e-8
    expect = anchor - (1 + eps) * np.array(v) - np.array([0.0, 0.0, m * g / k])
    assert np.abs(q[:3] - expect).max() < 1e-12
    A_expect = np.diag([1.0, 1.0, 1.0 + eps])
    assert np.abs(q[3:] - A_expect.T.reshape(-1)).max() < 1e-12
    assert np.abs(qd).max() < 1e-9


@pytest.mark.parametrize("theta", [0.7, -1.2])
def test_revolute_drive_reaches_target_angle(theta):
    # a 40 x 8 x 8 mm link hinged at its -x end on the world z axis (two point springs on the axis) and
    # driven by a direction spring from its x axis to (cos theta, sin theta, 0)
    L, w = 40 * MM, 8 * MM
    hinge = np.array([0.0, 0.0, 0.05])
    joints = [dict(a=0, a_kind=0, a_vec=(-L / 2, 0.0, s * w / 2), b=-1, b_kind=0, b_vec=(0, 0, 0), k=2e4,
                   t=tuple(hinge + [0.0, 0.0, s * w / 2])) for s in (-1.0, 1.0)]
    joints.append(dict(a=0, a_kind=1, a_vec=(1.0, 0.0, 0.0), b=-1, b_kind=1, b_vec=(0, 0, 0), k=1.0,
                       t=(math.cos(theta), math.sin(theta), 0.0)))
    sc = _scene([_box((L / 2, w / 2, w / 2), centre=hinge + [L / 2, 0.0, 0.0])], joints, n_steps=60)
    o = _run(sc)
    q, _ = _q(o, 0)
    c, s = math.cos(theta), math.sin(theta)
    R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    assert np.abs(q[3:] - R.T.reshape(-1)).max() < 1e-8
    assert np.abs(q[:3] - (hinge + R @ [L / 2, 0.0, 0.0])).max() < 1e-9


def test_prismatic_drive_slides_along_the_parent_axis():
    # body 1 (the parent) held by three world point springs at its corners; body 0 tied by a point spring
    # from its centre to the parent point (0, 0, 0) + s e_x (s per step, the b-side vector) and by three
    # direction springs to the parent's axes (orientation locked): p_0 = p_1 + A_1 (s, 0, 0)
    h = 5 * MM
    Rp = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])  # parent turned 90 deg about z
    cp = np.array([0.02, 0.01, 0.03])
    joints = []
    for v in ((h, h, h), (-h, h, -h), (h, -h, -h)):
        joints.append(dict(a=1, a_kind=0, a_vec=v, b=-1, b_kind=0, b_vec=(0, 0, 0), k=1e3,
                           t=tuple(cp + Rp @ np.array(v))))
    s0, s_final = 15 * MM, 32 * MM
    joints.append(dict(a=0, a_kind=0, a_vec=(0.0, 0.0, 0.0), b=1, b_kind=0, b_vec=(s0, 0.0, 0.0), k=50.0,
                       t=(0.0, 0.0, 0.0)))
    for e in np.eye(3):
        joints.append(dict(a=0, a_kind=1, a_vec=tuple(e), b=1, b_kind=1, b_vec=tuple(e), k=1.0, t=(0.0, 0.0, 0.0)))
    n = 60
    joint_b = np.array([[j["b_vec"] for j in joints]] * (n + 1), float)
    for k in range(n + 1):
        joint_b[k, 3] = (s0 + (s_final - s0) * min(1.0, k / 20), 0.0, 0.0)
    sc = _scene([_box((h, h, h), centre=cp + Rp @ [s0, 0.0, 0.0], A=Rp), _box((h, h, h), centre=cp, A=Rp)], joints,
                n_steps=n, joint_b=joint_b)
    o = _run(sc)
    q0, _ = _q(o, 0)
    q1, _ = _q(o, 1)
    assert np.abs(q1[:3] - cp).max() < 1e-9
    assert np.abs(q0[:3] - (cp + Rp @ [s_final, 0.0, 0.0])).max() < 1e-9
    assert np.abs(q0[3:] - Rp.T.reshape(-1)).max() < 1e-8


def test_joint_forces_conserve_linear_momentum():
    # two free boxes of different density joined by a stretched point spring between off-centre points, no
    # gravity: the joint force is internal, so sum_b m_b pdot_b stays zero while both move (and turn)
    h = 5 * MM
    joints = [dict(a=0, a_kind=0, a_vec=(h, 0.5 * h, 0.0), b=1, b_kind=0, b_vec=(-h, 0.0, -0.5 * h), k=5.0,
                   t=(0.0, 0.0, 0.0))]
    abd = [_box((h, h, h), rho=1000.0, centre=(0.0, 0.0, 0.0)), _box((h, h, h), rho=3000.0, centre=(0.03, 0.004, 0.0))]
    sc = _scene(abd, joints, n_steps=8)
    o = _run(sc)
    m = [1000.0 * (2 * h) ** 3, 3000.0 * (2 * h) ** 3]
    (_, qd0), (_, qd1) = _q(o, 0), _q(o, 1)
    P = m[0] * qd0[:3] + m[1] * qd1[:3]
    assert np.linalg.norm(qd0[:3]) > 1e-3 and np.linalg.norm(qd1[:3]) > 1e-4
    assert np.abs(P).max() < 1e-10 * m[0] * np.linalg.norm(qd0[:3])


def test_joint_energy_terms_match_the_definition_at_random_states():
    # E_joint from evaluate against the definition written with world points x = p + A v (directions A v)
    r = np.random.default_rng(3)
    h = 5 * MM
    joints = [dict(a=0, a_kind=0, a_vec=tuple(r.normal(size=3) * h), b=1, b_kind=0,
                   b_vec=tuple(r.normal(size=3) * h), k=7.0, t=tuple(r.normal(size=3) * 1e-3)),
              dict(a=1, a_kind=1, a_vec=tuple(r.normal(size=3)), b=0, b_kind=1, b_vec=tuple(r.normal(size=3)), k=0.3,
                   t=tuple(r.normal(size=3))),
              dict(a=0, a_kind=0, a_vec=tuple(r.normal(size=3) * h), b=-1, b_kind=0, b_vec=(0, 0, 0), k=2.0,
                   t=tuple(r.normal(size=3) * 1e-2))]
    abd = [_box((h, h, h), centre=(0.0, 0.0, 0.0)), _box((h, h, h), centre=(0.05, 0.0, 0.0))]
    sc = _scene(abd, joints, n_steps=1)
    S = ipc.Scene(sc)
    z = S.z0 + 1e-3 * r.normal(size=S.ndof)
    ctx = dict(z_tilde=z.copy(), x_t=S.positions(z), lag=[], stitch_hat=S.stitch_targets(1))
    E, _, _, info = S.evaluate(z, ctx, want_grad=False, want_hess=False)
    expect = 0.0
    for jn in joints:
        sides = []
        for body, kind, v in ((jn["a"], jn["a_kind"], jn["a_vec"]), (jn["b"], jn["b_kind"], jn["b_vec"])):
            if body < 0:
                sides.append(np.zeros(3))
                continue
            q = z[S.n_fem_dof + 12 * body:S.n_fem_dof + 12 * body + 12]
            A = np.stack([q[3:6], q[6:9], q[9:12]], axis=1)
            sides.append(A @ np.asarray(v) + (q[:3] if kind == 0 else 0.0))
        d = sides[0] - sides[1] - np.asarray(jn["t"])
        expect += 0.5 * jn["k"] * d @ d
    assert abs(info["E_joint"] - expect) <= 1e-12 * expect
