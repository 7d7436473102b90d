"""Plain FP64 CPU oracle for the IPC time step (Eq. 1-3, §III-C.1 and §III-C.2).

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
CPU-baseline leg of the benchmark may import this module.  It shares no code
with the CUDA library: the element, distance, barrier, friction and CCD
arithmetic is in ``ipc_oracle.cpp`` (plain loops), the Newton iteration and
all sparse assembly are here, and the linear solve is scipy's sparse direct
solver.

One step minimises the incremental potential of Eq. 3 over the free DOFs
(FEM vertices, ABD bodies) with kinematic bodies held at their prescribed
transforms (the arm links and finger bases follow prescribed rigid motions;
the bidirectional joint drive is not modelled):

  E(z) = 1/2 (z - z~)^T M (z - z~)
       + dt^2 [ sum_e V_e Psi(F_e)                   (E_FEM, §III-C.1)
              + kappa sum_k m_k b(s_k)               (E_barrier)
              + sum_k D_k                            (E_friction, lagged)
              + 1/2 k_c sum_i |x_i - x^_i|^2         (E_stitch, Eq. 2)
              + sum_A kappa_A V_A |A^T A - I|_F^2 ]  (E_ABD)

DOF vector z = [FEM vertex positions (3 each) | ABD q = (p, A columns)
(12 each) | kinematic vertex positions (3 each)].  Every vertex position is
linear in z: x = Jmap z (identity for FEM and kinematic vertices,
x = p + A xbar for ABD surface vertices).
"""
from __future__ import annotations

import ctypes as C
import math
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import build as _build

_lib = None
dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int)


class OrcSurf(C.Structure):
    _fields_ = [("nsv", C.c_int), ("ntri", C.c_int), ("nedge", C.c_int),
                ("sv", ip), ("tri", ip), ("edge", ip), ("vbody", ip), ("bkind", ip)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        L = _lib
        L.orc_snh.argtypes = [dp, C.c_double, C.c_double, C.c_int, dp, dp, dp]
        L.orc_tet.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double, C.c_int, dp, dp, dp]
        L.orc_elastic_all.argtypes = [C.c_int, ip, dp, dp, dp, dp, dp, C.c_int, dp, dp, dp]
        L.orc_pt_dist.argtypes = [dp, C.c_int, dp, dp, dp]
        L.orc_ee_dist.argtypes = [dp, C.c_int, dp, dp, dp]
        L.orc_pt_classify.argtypes = [dp, dp, dp]
        L.orc_pt_classify.restype = C.c_int
        L.orc_ee_classify.argtypes = [dp, dp, dp]
        L.orc_ee_classify.restype = C.c_int
        L.orc_barrier.argtypes = [C.c_double, C.c_double, dp, dp, dp]
        L.orc_ee_mollifier.argtypes = [dp, C.c_double, dp, dp, dp]
        L.orc_pair.argtypes = [C.c_int, C.c_int, dp, C.c_double, C.c_double, C.c_double, C.c_int, dp, dp, dp]
        L.orc_friction.argtypes = [dp, dp, C.c_double, C.c_double, C.c_double, dp, dp, dp, dp, dp]
        L.orc_active_pairs.argtypes = [C.POINTER(OrcSurf), dp, C.c_double, C.c_int, ip, dp]
        L.orc_active_pairs.restype = C.c_int
        L.orc_accd.argtypes = [C.c_int, dp, dp, C.c_double, C.c_double, C.c_int]
        L.orc_accd.restype = C.c_double
        L.orc_ccd_alpha.argtypes = [C.POINTER(OrcSurf), dp, dp, C.c_double, C.c_int, ip]
        L.orc_ccd_alpha.restype = C.c_double
        L.orc_abd_orth.argtypes = [dp, C.c_double, C.c_int, dp, dp, dp]
        L.orc_project_psd.argtypes = [C.c_int, dp]
        L.orc_jacobi_eigen.argtypes = [C.c_int, dp, dp]
        L.orc_jacobi_eigen.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_get_threads.restype = C.c_int
    return _lib


def set_threads(n: int):
    """Threads of the brute-force pair loops (results do not depend on it); <= 0: all cores."""
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def _d(a):
    return a.ctypes.data_as(dp)


def _i(a):
    return a.ctypes.data_as(ip)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ----------------------------------------------------------------------------
# per-primitive wrappers (used directly by the pin tests)
# ----------------------------------------------------------------------------

def snh(F, mu, lam, project=False):
    """Psi, P (3x3), d2Psi/dvec(F)^2 (9x9, vec column-major) for one F."""
    F = _f64(F).reshape(9)
    psi = C.c_double()
    P = np.zeros(9)
    H = np.zeros(81)
    lib().orc_snh(_d(F), mu, lam, int(project), C.byref(psi), _d(P), _d(H))
    return psi.value, P.reshape(3, 3), H.reshape(9, 9)


def tet(x, B, vol, mu, lam, project=False):
    x = _f64(x).reshape(12)
    B = _f64(B).reshape(9)
    E = C.c_double()
    g = np.zeros(12)
    H = np.zeros(144)
    lib().orc_tet(_d(x), _d(B), vol, mu, lam, int(project), C.byref(E), _d(g), _d(H))
    return E.value, g, H.reshape(12, 12)


def pt_dist(x, type_):
    x = _f64(x).reshape(12)
    s = C.c_double()
    g = np.zeros(12)
    H = np.zeros(144)
    lib().orc_pt_dist(_d(x), int(type_), C.byref(s), _d(g), _d(H))
    return s.value, g, H.reshape(12, 12)


def ee_dist(x, type_):
    x = _f64(x).reshape(12)
    s = C.c_double()
    g = np.zeros(12)
    H = np.zeros(144)
    lib().orc_ee_dist(_d(x), int(type_), C.byref(s), _d(g), _d(H))
    return s.value, g, H.reshape(12, 12)


def classify(kind, x):
    """(type, s, closest-point weights w) of a point-triangle (0) or edge-edge (1) stencil."""
    x = _f64(x).reshape(12)
    s = C.c_double()
    w = np.zeros(4)
    f = lib().orc_pt_classify if kind == 0 else lib().orc_ee_classify
    t = f(_d(x), C.byref(s), _d(w))
    return t, s.value, w


def barrier(s, sh):
    b, b1, b2 = C.c_double(), C.c_double(), C.c_double()
    lib().orc_barrier(float(s), float(sh), C.byref(b), C.byref(b1), C.byref(b2))
    return b.value, b1.value, b2.value


def ee_mollifier(x, eps_x):
    x = _f64(x).reshape(12)
    m = C.c_double()
    g = np.zeros(12)
    H = np.zeros(144)
    lib().orc_ee_mollifier(_d(x), float(eps_x), C.byref(m), _d(g), _d(H))
    return m.value, g, H.reshape(12, 12)


def pair(kind, type_, x, sh, kappa, eps_x, project=False):
    x = _f64(x).reshape(12)
    E = C.c_double()
    g = np.zeros(12)
    H = np.zeros(144)
    lib().orc_pair(int(kind), int(type_), _d(x), float(sh), float(kappa), float(eps_x), int(project),
                   C.byref(E), _d(g), _d(H))
    return E.value, g, H.reshape(12, 12)


def friction(w, n, lam, mu, eps, x, xt):
    w = _f64(w); n = _f64(n); x = _f64(x).reshape(12); xt = _f64(xt).reshape(12)
    E = C.c_double()
    g = np.zeros(12)
    H = np.zeros(144)
    lib().orc_friction(_d(w), _d(n), float(lam), float(mu), float(eps), _d(x), _d(xt), C.byref(E), _d(g), _d(H))
    return E.value, g, H.reshape(12, 12)


def accd(kind, x, p, s_frac=0.1, tmax=1.0, max_iter=1_000_000):
    x = _f64(x).reshape(12)
    p = _f64(p).reshape(12)
    return lib().orc_accd(int(kind), _d(x), _d(p), float(s_frac), float(tmax), int(max_iter))


def abd_orth(a, k, project=False):
    a = _f64(a).reshape(9)
    E = C.c_double()
    g = np.zeros(9)
    H = np.zeros(81)
    lib().orc_abd_orth(_d(a), float(k), int(project), C.byref(E), _d(g), _d(H))
    return E.value, g, H.reshape(9, 9)


def project_psd(H):
    n = H.shape[0]
    A = _f64(H).copy().reshape(-1)
    lib().orc_project_psd(n, _d(A))
    return A.reshape(n, n)


def jacobi_eigen(H):
    n = H.shape[0]
    A = _f64(H).copy().reshape(-1)
    V = np.zeros(n * n)
    lib().orc_jacobi_eigen(n, _d(A), _d(V))
    return np.diag(A.reshape(n, n)).copy(), V.reshape(n, n)


def snh_params(E, nu):
    """Model parameters (mu, lam_model) of the Neo-Hookean form from Young's
    modulus E and Poisson ratio nu (§III-C.1 specifies the material by E, nu).

    mu/2 (tr F^T F - 3) - mu (J - 1) + lam_model/2 (J - 1)^2 linearises at
    F = I to mu eps:eps + (lam_model - mu)/2 tr(eps)^2, so lam_model =
    lam + mu (lam the first Lame parameter) makes its small-strain limit the
    linear material with exactly E and nu."""
    mu = E / (2 * (1 + nu))
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    return mu, lam + mu


# ----------------------------------------------------------------------------
# barrier stiffness: kappa = kbar / B''(dhat / 2), B(d) = b(d^2)
# ----------------------------------------------------------------------------

def barrier_d2_dist(d, dhat):
    """d^2/dd^2 of b(d^2) with kappa = 1: 4 d^2 b''(s) + 2 b'(s), s = d^2."""
    sh = dhat * dhat
    s = d * d
    dd = s - sh
    l = math.log(s / sh)
    b1 = -(2 * dd * l + dd * dd / s)
    b2 = -(2 * l + 4 * dd / s - dd * dd / (s * s))
    return 4 * s * b2 + 2 * b1


# ----------------------------------------------------------------------------
# scene preparation
# ----------------------------------------------------------------------------

def _tet_faces_outward(tets):
    t = tets
    return np.concatenate([t[:, [1, 2, 3]], t[:, [0, 3, 2]], t[:, [0, 1, 3]], t[:, [0, 2, 1]]], axis=0)


def extract_surface(tets):
    """Faces that belong to exactly one tet, outward oriented."""
    faces = _tet_faces_outward(tets)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    inv = inv.reshape(-1)
    return faces[cnt[inv] == 1].astype(np.int32)


def tri_edges(tris):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    return np.unique(e, axis=0).astype(np.int32)


def closed_mesh_moments(X, tris):
    """Volume integrals of 1, x_i and x_i x_j over a closed outward mesh.

    Each triangle with the origin spans a signed tet of volume det[a,b,c]/6;
    over a tet with vertices v_k, int x = V/4 sum v_k and
    int x x^T = V/20 (sum v_k v_k^T + (sum v_k)(sum v_k)^T)."""
    a, b, c = X[tris[:, 0]], X[tris[:, 1]], X[tris[:, 2]]
    V = np.einsum("ij,ij->i", a, np.cross(b, c)) / 6.0
    vol = V.sum()
    ssum = a + b + c
    first = (V[:, None] * ssum / 4.0).sum(0)
    outer = (np.einsum("ni,nj->nij", a, a) + np.einsum("ni,nj->nij", b, b) + np.einsum("ni,nj->nij", c, c)
             + np.einsum("ni,nj->nij", ssum, ssum))
    second = (V[:, None, None] * outer / 20.0).sum(0)
    return vol, first, second


class Scene:
    """Mesh preparation and the DOF map for one scene dictionary."""

    def __init__(self, sc: dict):
        self.sc = sc
        P = sc["params"]
        self.dt = P["dt"]
        self.dhat = P["dhat"]
        self.sh = self.dhat * self.dhat
        self.mu_f = P["mu"]
        self.eps = P["eps_v"] * self.dt
        self.tol = P["newton_tol"]
        self.max_newton = int(P["max_newton"])
        self.s_ccd = P["s_ccd"]
        self.kappa_A = P["kappa_A"]
        self.g = _f64(sc["gravity"])

        # FEM ------------------------------------------------------------
        X = _f64(sc["fem_X"])
        T = _i32(sc["fem_tets"])
        self.nf = X.shape[0]
        self.tets = T
        Dm = np.stack([X[T[:, 1]] - X[T[:, 0]], X[T[:, 2]] - X[T[:, 0]], X[T[:, 3]] - X[T[:, 0]]], axis=-1)
        vol = np.linalg.det(Dm) / 6.0
        if np.any(vol <= 0):
            raise ValueError("inverted or degenerate rest tetrahedron")
        self.vol = vol
        self.B = np.ascontiguousarray(np.linalg.inv(Dm).reshape(-1, 9))
        self.nu = _f64(sc["fem_nu"])
        self.logE = _f64(sc["fem_logE"]).copy()
        self.mu, self.lam = snh_params(np.exp(self.logE), self.nu)
        rho = _f64(sc["fem_rho"])
        self.mass_v = np.zeros(self.nf)
        np.add.at(self.mass_v, T.reshape(-1), np.repeat(rho * vol / 4.0, 4))
        fem_surf = extract_surface(T)
        fem_vbody = np.zeros(self.nf, np.int32)
        fb = _i32(sc.get("fem_body", np.zeros(len(T), np.int32)))
        fem_vbody[T.reshape(-1)] = np.repeat(fb, 4)
        n_fem_bodies = int(fb.max()) + 1 if len(fb) else 0

        # ABD ------------------------------------------------------------
        abd = sc.get("abd", [])
        self.nab = len(abd)
        self.abd_S = []
        self.abd_vol = []
        abd_X, abd_tris, abd_off = [], [], []
        off = self.nf
        for A in abd:
            vol_a, first, second = closed_mesh_moments(_f64(A["X"]), _i32(A["tris"]))
            rho_a = A["rho"]
            S = np.zeros((4, 4))
            S[0, 0] = vol_a
            S[0, 1:] = first
            S[1:, 0] = first
            S[1:, 1:] = second
            self.abd_S.append(rho_a * S)
            self.abd_vol.append(vol_a)
            abd_X.append(_f64(A["X"]))
            abd_tris.append(_i32(A["tris"]) + off)
            abd_off.append(off)
            off += A["X"].shape[0]
        self.na_v = off - self.nf

        # kinematic ------------------------------------------------------
        kin = sc.get("kin", [])
        self.nkb = len(kin)
        kin_tris, kin_off = [], []
        for K in kin:
            kin_tris.append(_i32(K["tris"]) + off)
            kin_off.append(off)
            off += K["X"].shape[0]
        self.nk = off - self.nf - self.na_v
        self.nv = off
        self.kin_off = kin_off
        self.abd_off = abd_off

        # bodies: FEM bodies, then ABD, then kinematic
        vbody = np.zeros(self.nv, np.int32)
        vbody[:self.nf] = fem_vbody
        bkind = [0] * n_fem_bodies
        for i, A in enumerate(abd):
            vbody[abd_off[i]:abd_off[i] + A["X"].shape[0]] = len(bkind)
            bkind.append(1)
        for i, K in enumerate(kin):
            vbody[kin_off[i]:kin_off[i] + K["X"].shape[0]] = len(bkind)
            bkind.append(2)
        self.vbody = vbody
        self.bkind = np.asarray(bkind, np.int32)

        # contact surface --------------------------------------------------
        tris = np.concatenate([fem_surf] + abd_tris + kin_tris, axis=0).astype(np.int32)
        self.tris = tris
        self.edges = tri_edges(tris) if len(tris) else np.zeros((0, 2), np.int32)
        self.sv = np.unique(tris.reshape(-1)).astype(np.int32)
        # rest positions of every vertex (for edge rest lengths and ABD maps)
        Xrest = np.zeros((self.nv, 3))
        Xrest[:self.nf] = X
        for i, A in enumerate(abd):
            Xrest[abd_off[i]:abd_off[i] + A["X"].shape[0]] = A["X"]
        for i, K in enumerate(kin):
            Xrest[kin_off[i]:kin_off[i] + K["X"].shape[0]] = K["X"]
        self.Xrest = Xrest
        el = Xrest[self.edges[:, 0]] - Xrest[self.edges[:, 1]]
        self.edge_rest_sq = np.einsum("ij,ij->i", el, el)
        self._edge_index = {(int(a), int(b)): k for k, (a, b) in enumerate(self.edges)}
        self.surf = OrcSurf(len(self.sv), len(self.tris), len(self.edges), _i(self.sv), _i(self.tris),
                            _i(self.edges), _i(self.vbody), _i(self.bkind))

        # DOFs -------------------------------------------------------------
        self.n_fem_dof = 3 * self.nf
        self.n_abd_dof = 12 * self.nab
        self.n_free = self.n_fem_dof + self.n_abd_dof
        self.ndof = self.n_free + 3 * self.nk
        rows, cols, vals = [], [], []
        r = np.arange(3 * self.nf)
        rows.append(r); cols.append(r); vals.append(np.ones(3 * self.nf))
        for i, A in enumerate(abd):
            n = A["X"].shape[0]
            xb = _f64(A["X"])
            base_r = 3 * abd_off[i]
            base_c = self.n_fem_dof + 12 * i
            for v in range(n):
                phi = (1.0, xb[v, 0], xb[v, 1], xb[v, 2])
                for k in range(4):
                    for d in range(3):
                        rows.append(np.array([base_r + 3 * v + d]))
                        cols.append(np.array([base_c + 3 * k + d]))
                        vals.append(np.array([phi[k]]))
        rk = np.arange(3 * self.nk)
        rows.append(3 * (self.nf + self.na_v) + rk)
        cols.append(self.n_free + rk)
        vals.append(np.ones(3 * self.nk))
        self.Jmap = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                                  shape=(3 * self.nv, self.ndof))

        # mass matrix in DOF space
        mr, mc, mv = [np.arange(3 * self.nf)], [np.arange(3 * self.nf)], [np.repeat(self.mass_v, 3)]
        for i in range(self.nab):
            S = self.abd_S[i]
            base = self.n_fem_dof + 12 * i
            for a in range(4):
                for b in range(4):
                    for d in range(3):
                        mr.append(np.array([base + 3 * a + d]))
                        mc.append(np.array([base + 3 * b + d]))
                        mv.append(np.array([S[a, b]]))
        self.M = sp.csr_matrix((np.concatenate(mv), (np.concatenate(mr), np.concatenate(mc))),
                               shape=(self.ndof, self.ndof))
        # gravity acceleration in DOF space: every FEM vertex, and the translation of every ABD body
        ga = np.zeros(self.ndof)
        ga[:self.n_fem_dof] = np.tile(self.g, self.nf)
        for i in range(self.nab):
            ga[self.n_fem_dof + 12 * i:self.n_fem_dof + 12 * i + 3] = self.g
        self.grav_acc = ga

        # elastic Hessian scatter indices (tet-major 12x12 blocks)
        dof = (3 * T[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 12)
        self.el_rows = np.repeat(dof, 12, axis=1).reshape(-1)
        self.el_cols = np.tile(dof, (1, 12)).reshape(-1)

        # stitch springs (Eq. 2)
        self.stitch_v = _i32(sc.get("stitch_v", np.zeros(0, np.int32)))
        self.stitch_b = _i32(sc.get("stitch_b", np.zeros(0, np.int32)))
        self.stitch_X = _f64(sc.get("stitch_X", np.zeros((0, 3))))

        # joints between affine bodies (E_joint of Eq. 3): quadratic springs
        # 1/2 k |J_a(abar) q_a - J_b(bbar) q_b - t|^2, where J(v) = [I, v0 I, v1 I, v2 I] maps a body-frame
        # point v to world (x = p + A v) and [0, v0 I, v1 I, v2 I] a body-frame direction; body b = -1 is
        # the world (its term vanishes, t is the world anchor)
        jn = sc.get("joints", [])
        self.n_joints = len(jn)
        self.joint_body = np.array([[j["a"], j["b"]] for j in jn], np.int64).reshape(-1, 2)
        self.joint_kind = np.array([[j["a_kind"], j["b_kind"]] for j in jn], np.int64).reshape(-1, 2)
        self.joint_vec = np.array([[j["a_vec"], j["b_vec"]] for j in jn], np.float64).reshape(-1, 2, 3)
        self.joint_k = np.array([j["k"] for j in jn], np.float64)
        self.joint_t = np.array([j.get("t", (0.0, 0.0, 0.0)) for j in jn], np.float64).reshape(-1, 3)

        # scalar parameters fixed at creation -----------------------------
        surf_fem_edges = self.edges[(self.edges[:, 0] < self.nf) & (self.edges[:, 1] < self.nf)]
        if len(surf_fem_edges):
            d = Xrest[surf_fem_edges[:, 0]] - Xrest[surf_fem_edges[:, 1]]
            ell = float(np.mean(np.sqrt(np.einsum("ij,ij->i", d, d))))
        elif len(vol):
            ell = float(np.mean(np.cbrt(vol)))
        else:
            ell = self.dhat  # no deformable body: the automatic stiffnesses use dhat and E = 1e5 Pa
        Emax = float(np.exp(np.max(sc["fem_logE"]))) if len(sc["fem_logE"]) else 1e5
        self.kappa = P["kappa"] if P["kappa"] > 0 else Emax * ell / barrier_d2_dist(0.5 * self.dhat, self.dhat)
        # adaptive barrier stiffness (IPC's kappa growth): after a Newton iteration whose iterate had its
        # smallest distance below kappa_dmin * dhat without that distance having grown since the step's
        # previous iterate, kappa doubles, up to kappa_max_factor times its initial value
        self.kappa_adaptive = bool(P.get("kappa_adaptive", 0))
        self.kappa_dmin = float(P.get("kappa_dmin", 1e-2))
        self.kappa_max = self.kappa * float(P.get("kappa_max_factor", 100.0))
        self.k_c = P["k_c"] if P["k_c"] > 0 else 100.0 * Emax * ell
        free_pts = [X]
        for i, A in enumerate(abd):
            q0 = _f64(A["q0"])
            Am = np.stack([q0[3:6], q0[6:9], q0[9:12]], axis=1)
            free_pts.append(_f64(A["X"]) @ Am.T + q0[:3])
        fp = np.concatenate(free_pts, 0)
        self.L = float(np.linalg.norm(fp.max(0) - fp.min(0)))

        # initial state
        z = np.zeros(self.ndof)
        z[:self.n_fem_dof] = X.reshape(-1)
        for i, A in enumerate(abd):
            z[self.n_fem_dof + 12 * i:self.n_fem_dof + 12 * (i + 1)] = _f64(A["q0"])
        z[self.n_free:] = self.kin_positions(0)
        self.z0 = z
        zd = np.zeros(self.ndof)
        if "fem_V0" in sc:
            zd[:self.n_fem_dof] = _f64(sc["fem_V0"]).reshape(-1)
        self.zd0 = zd

    # ------------------------------------------------------------------
    def kin_positions(self, step):
        out = np.zeros(3 * self.nk)
        Ts = self.sc["kin_T"][step] if self.nkb else None
        o = 0
        for i, K in enumerate(self.sc.get("kin", [])):
            n = K["X"].shape[0]
            Tm = Ts[i]
            out[3 * o:3 * (o + n)] = (_f64(K["X"]) @ Tm[:, :3].T + Tm[:, 3]).reshape(-1)
            o += n
        return out

    def joint_targets(self, step):
        """The joints' b-side vectors and targets of step `step` (scene keys joint_b / joint_t, per step)."""
        out = {}
        if self.n_joints and "joint_b" in self.sc:
            out["joint_b"] = _f64(self.sc["joint_b"][step])
        if self.n_joints and "joint_t" in self.sc:
            out["joint_t"] = _f64(self.sc["joint_t"][step])
        return out

    def stitch_targets(self, step):
        if len(self.stitch_v) == 0:
            return np.zeros((0, 3))
        Ts = self.sc["kin_T"][step]
        out = np.zeros((len(self.stitch_v), 3))
        for k in range(len(self.stitch_v)):
            Tm = Ts[self.stitch_b[k]]
            out[k] = Tm[:, :3] @ self.stitch_X[k] + Tm[:, 3]
        return out

    def positions(self, z):
        return (self.Jmap @ z).reshape(-1, 3)

    # ------------------------------------------------------------------
    # contact
    # ------------------------------------------------------------------
    def active_pairs(self, x):
        """Brute-force active set: list of records (kind, prim_a, prim_b, type, v0..v3) and s."""
        x = _f64(x)
        cap = 4096
        while True:
            rec = np.zeros((cap, 8), np.int32)
            s = np.zeros(cap)
            n = lib().orc_active_pairs(C.byref(self.surf), _d(x), self.sh, cap, _i(rec), _d(s))
            if n <= cap:
                return rec[:n].copy(), s[:n].copy()
            cap = n

    def eps_x(self, rec):
        """Mollifier threshold 1e-3 |ea_rest|^2 |eb_rest|^2 for each edge-edge record."""
        out = np.zeros(len(rec))
        m = rec[:, 0] == 1
        out[m] = 1e-3 * self.edge_rest_sq[rec[m, 1]] * self.edge_rest_sq[rec[m, 2]]
        return out

    def friction_lag(self, x):
        """Lagged friction data at the start of the step: per active pair the
        closest-point weights w, unit normal n and normal force lambda."""
        x = _f64(x).reshape(-1, 3)
        rec, s = self.active_pairs(x.reshape(-1))
        epsx = self.eps_x(rec)
        lag = []
        for k in range(len(rec)):
            kind = int(rec[k, 0])
            ids = rec[k, 4:8]
            xs = x[ids]
            t, sk, w = classify(kind, xs)
            d = math.sqrt(sk)
            nvec = (w[:, None] * xs).sum(0) / d
            _, b1, _ = barrier(sk, self.sh)
            m = ee_mollifier(xs, epsx[k])[0] if kind == 1 else 1.0
            lam = -self.kappa * m * 2.0 * d * b1
            lag.append((ids.copy(), w, nvec, lam))
        return lag

    # ------------------------------------------------------------------
    # energy, gradient, Hessian of the incremental potential
    # ------------------------------------------------------------------
    def evaluate(self, z, ctx, want_grad=True, want_hess=True, project=True):
        """Returns (E, g, H, info) in DOF space.  ctx holds z~, x_t, lag, stitch targets."""
        dt2 = self.dt * self.dt
        x = self.positions(z)
        xf = x.reshape(-1)
        nvd = 3 * self.nv
        # inertia
        dz = z - ctx["z_tilde"]
        Mdz = self.M @ dz
        E_in = 0.5 * float(dz @ Mdz)
        g = Mdz.copy() if want_grad else None
        Hrows, Hcols, Hvals = [], [], []
        # elastic
        Eel = C.c_double(0.0)
        gv = np.zeros(nvd)
        Hv = np.zeros(len(self.tets) * 144) if want_hess else None
        lib().orc_elastic_all(len(self.tets), _i(self.tets), _d(self.B), _d(self.vol), _d(self.mu), _d(self.lam),
                              _d(xf), int(project), C.byref(Eel), _d(gv),
                              _d(Hv) if want_hess else C.cast(0, dp))
        E_pot = Eel.value
        if want_hess:
            Hrows.append(self.el_rows); Hcols.append(self.el_cols); Hvals.append(Hv)
        # barrier on the current active set
        rec, s = self.active_pairs(xf)
        epsx = self.eps_x(rec)
        E_bar = 0.0
        for k in range(len(rec)):
            kind, _, _, t = (int(v) for v in rec[k, :4])
            ids = rec[k, 4:8]
            Ek, gk, Hk = pair(kind, t, x[ids], self.sh, self.kappa, epsx[k], project)
            E_bar += Ek
            dofs = (3 * ids[:, None] + np.arange(3)).reshape(-1)
            np.add.at(gv, dofs, gk)
            if want_hess:
                Hrows.append(np.repeat(dofs, 12)); Hcols.append(np.tile(dofs, 12)); Hvals.append(Hk.reshape(-1))
        # friction on the lagged pairs
        E_fr = 0.0
        if self.mu_f > 0:
            xt = ctx["x_t"]
            for ids, w, nvec, lam in ctx["lag"]:
                Ek, gk, Hk = friction(w, nvec, lam, self.mu_f, self.eps, x[ids], xt[ids])
                E_fr += Ek
                dofs = (3 * ids[:, None] + np.arange(3)).reshape(-1)
                np.add.at(gv, dofs, gk)
                if want_hess:
                    Hrows.append(np.repeat(dofs, 12)); Hcols.append(np.tile(dofs, 12)); Hvals.append(Hk.reshape(-1))
        # stitch springs
        E_st = 0.0
        if len(self.stitch_v):
            d = x[self.stitch_v] - ctx["stitch_hat"]
            E_st = 0.5 * self.k_c * float((d * d).sum())
            dofs = (3 * self.stitch_v[:, None] + np.arange(3)).reshape(-1)
            np.add.at(gv, dofs, self.k_c * d.reshape(-1))
            if want_hess:
                Hrows.append(dofs); Hcols.append(dofs); Hvals.append(np.full(len(dofs), self.k_c))
        total_pot = E_pot + E_bar + E_fr + E_st
        # vertex space -> DOF space
        if want_grad:
            g += dt2 * (self.Jmap.T @ gv)
        H = None
        if want_hess:
            Hvert = sp.csr_matrix((np.concatenate(Hvals), (np.concatenate(Hrows), np.concatenate(Hcols))),
                                  shape=(nvd, nvd))
            H = self.M + dt2 * (self.Jmap.T @ Hvert @ self.Jmap)
        # ABD orthogonality in DOF space
        E_abd = 0.0
        for i in range(self.nab):
            base = self.n_fem_dof + 12 * i
            k = self.kappa_A * self.abd_vol[i]
            Ea, ga, Ha = abd_orth(z[base + 3:base + 12], k, project)
            E_abd += Ea
            if want_grad:
                g[base + 3:base + 12] += dt2 * ga
            if want_hess:
                idx = np.arange(base + 3, base + 12)
                H = H + sp.csr_matrix((dt2 * Ha.reshape(-1), (np.repeat(idx, 9), np.tile(idx, 9))),
                                      shape=(self.ndof, self.ndof))
        # joints (E_joint): the drive directions of this step come from ctx["joint_b"] when given
        E_jt = 0.0
        if self.n_joints:
            G, t = self.joint_operator(ctx.get("joint_b"), ctx.get("joint_t"))
            r = G @ z - t
            kk = np.repeat(self.joint_k, 3)
            E_jt = 0.5 * float(r @ (kk * r))
            if want_grad:
                g = g + dt2 * (G.T @ (kk * r))
            if want_hess:
                H = H + dt2 * (G.T @ sp.diags(kk) @ G)
        E = E_in + dt2 * (total_pot + E_abd + E_jt)
        info = dict(n_pairs=len(rec), min_s=float(s.min()) if len(s) else math.inf,
                    E_inertia=E_in, E_elastic=E_pot, E_barrier=E_bar, E_friction=E_fr, E_stitch=E_st, E_abd=E_abd,
                    E_joint=E_jt)
        return E, g, H, info

    def joint_operator(self, joint_b=None, joint_t=None):
        """G (3 n_joints x ndof) and t with r_j = (G z - t)_j = J_a q_a - J_b q_b - t_j for every joint."""
        rows, cols, vals = [], [], []
        for j in range(self.n_joints):
            for side, sign in ((0, 1.0), (1, -1.0)):
                body = int(self.joint_body[j, side])
                if body < 0:
                    continue
                v = self.joint_vec[j, side] if (side == 0 or joint_b is None) else _f64(joint_b[j])
                w = (0.0 if self.joint_kind[j, side] == 1 else 1.0, v[0], v[1], v[2])
                base = self.n_fem_dof + 12 * body
                for m in range(4):
                    for d in range(3):
                        rows.append(3 * j + d)
                        cols.append(base + 3 * m + d)
                        vals.append(sign * w[m])
        G = sp.csr_matrix((vals, (rows, cols)), shape=(3 * self.n_joints, self.ndof))
        t = (self.joint_t if joint_t is None else _f64(joint_t)).reshape(-1)
        return G, t

    def energy(self, z, ctx):
        return self.evaluate(z, ctx, want_grad=False, want_hess=False)[0]

    def ccd_alpha(self, z, p):
        x = _f64(self.positions(z).reshape(-1))
        pv = _f64(self.Jmap @ p)
        nc = C.c_int()
        a = lib().orc_ccd_alpha(C.byref(self.surf), _d(x), _d(pv), self.s_ccd, ACCD_MAX_ITER, C.byref(nc))
        return a, nc.value


# Conservative-advancement iterations per candidate before ACCD returns the
# time reached so far (still a safe bound).
ACCD_MAX_ITER = 10000


class StepError(RuntimeError):
    pass


class Oracle:
    """State (z, zdot) and the time step."""

    def __init__(self, sc: dict, tol: float | None = None):
        self.S = Scene(sc)
        if tol is not None:
            self.S.tol = tol
        self.z = self.S.z0.copy()
        self.zd = self.S.zd0.copy()
        self.step_index = 0
        self.stats = []

    def x(self):
        return self.S.positions(self.z)

    def step(self, record_iterates=False):
        """One incremental-potential minimisation (Eq. 3) from z_t to z_{t+1}."""
        S = self.S
        t1 = self.step_index + 1
        z_t = self.z.copy()
        z = z_t.copy()
        z_tilde = z_t + S.dt * self.zd + S.dt * S.dt * S.grav_acc
        x_t = S.positions(z_t)
        ctx = dict(z_tilde=z_tilde, x_t=x_t, lag=S.friction_lag(x_t.reshape(-1)) if S.mu_f > 0 else [],
                   stitch_hat=S.stitch_targets(t1), **S.joint_targets(t1))
        zD_hat = S.kin_positions(t1)
        F = slice(0, S.n_free)
        D = slice(S.n_free, S.ndof)
        it_stats = []
        converged = False
        s_prev = math.inf  # smallest squared distance of the previous iterate (adaptive kappa)
        for it in range(S.max_newton):
            E, g, H, info = S.evaluate(z, ctx)
            pD = zD_hat - z[D]
            H = H.tocsr()
            HFF = H[F, F].tocsc()
            rhs = -g[F]
            if S.nk and np.any(pD != 0):
                rhs = rhs - H[F, D] @ pD
            pF = spla.spsolve(HFF, rhs) if S.n_free else np.zeros(0)
            p = np.concatenate([pF, pD])
            dirichlet_done = not np.any(pD != 0)
            pnorm = float(np.max(np.abs(pF))) if S.n_free else 0.0
            rec = dict(it=it, E=E, pnorm=pnorm / (S.dt * S.L), min_s=info["min_s"], n_pairs=info["n_pairs"])
            if dirichlet_done and pnorm <= S.tol * S.dt * S.L:
                converged = True
                it_stats.append(rec)
                break
            alpha, ncand = S.ccd_alpha(z, p)
            rec["alpha_ccd"] = alpha
            rec["n_ccd"] = ncand
            if dirichlet_done:
                # backtracking on the incremental potential; tolerance covers rounding of E
                n_half = 0
                stationary = False
                while True:
                    E_new = S.energy(z + alpha * p, ctx)
                    if E_new <= E + 1e-13 * abs(E):
                        break
                    alpha *= 0.5
                    n_half += 1
                    if alpha * pnorm <= S.tol * S.dt * S.L:
                        # no decrease resolvable above rounding within the tolerance: stationary
                        stationary = True
                        break
                    if n_half > 40:
                        raise StepError("line search stalled")
                if stationary:
                    converged = True
                    rec["stationary"] = True
                    it_stats.append(rec)
                    break
                rec["E_new"] = E_new
            z = z + alpha * p
            if alpha == 1.0:
                z[D] = zD_hat
            rec["alpha"] = alpha
            if S.kappa_adaptive:
                s_it = info["min_s"]
                if s_it < (S.kappa_dmin * S.dhat) ** 2 and s_it <= s_prev:
                    S.kappa = min(2.0 * S.kappa, S.kappa_max)
                s_prev = s_it
            rec["kappa"] = S.kappa
            it_stats.append(rec)
            if record_iterates:
                rec["z"] = z.copy()
        if not converged:
            raise StepError("Newton did not converge")
        self.zd = (z - z_t) / S.dt
        self.zd[D] = 0.0
        self.z = z
        self.step_index = t1
        self.stats.append(it_stats)
        return it_stats


# ----------------------------------------------------------------------------
# implicit adjoint of one step (dense)
# ----------------------------------------------------------------------------

def set_material(o: "Oracle", logE=None, mu=None):
    """Per-tet log Young's modulus and the friction coefficient used by later steps."""
    S = o.S
    if logE is not None:
        S.logE = _f64(logE).copy()
        S.mu, S.lam = snh_params(np.exp(S.logE), S.nu)
    if mu is not None:
        S.mu_f = float(mu)


def step_context(S, z_t, zd_t, step_next):
    x_t = S.positions(z_t)
    ctx = dict(z_tilde=z_t + S.dt * zd_t + S.dt * S.dt * S.grav_acc, x_t=x_t, lag=[], lag_kind=[], lag_eps_x=[],
               stitch_hat=S.stitch_targets(step_next), **S.joint_targets(step_next))
    if S.mu_f > 0:
        rec, _ = S.active_pairs(x_t.reshape(-1))
        ctx["lag"] = S.friction_lag(x_t.reshape(-1))
        ctx["lag_kind"] = [int(k) for k in rec[:, 0]]
        ctx["lag_eps_x"] = list(S.eps_x(rec))
    return ctx


def _free_weight_directions(kind, type_):
    """Directions (4, k) along which the closest-point weights of a distance type move: w = w0 + B theta
    with theta the type's free parameters (segment or barycentric coordinates); k = 0 for point-point."""
    if kind == 0:
        if type_ <= 2:
            return np.zeros((4, 0))
        if type_ <= 5:  # point against edge (t_k, t_k+1): w = e_p - (1 - t) e_k - t e_k+1
            k = type_ - 3
            B = np.zeros((4, 1))
            B[1 + k, 0], B[1 + (k + 1) % 3, 0] = 1.0, -1.0
            return B
        return np.array([[0.0, 0.0], [1.0, 1.0], [-1.0, 0.0], [0.0, -1.0]])  # w = [1, -(1-b1-b2), -b1, -b2]
    if type_ <= 3:
        return np.zeros((4, 0))
    if type_ <= 5:  # a point of edge b against edge a: w = [(1 - t), t, -1 (at that point)]
        return np.array([[-1.0], [1.0], [0.0], [0.0]])
    if type_ <= 7:  # a point of edge a against edge b: w = [1 (at that point), -(1 - t), -t]
        return np.array([[0.0], [0.0], [1.0], [-1.0]])
    return np.array([[-1.0, 0.0], [1.0, 0.0], [0.0, 1.0], [0.0, -1.0]])  # line-line (s, t)


def friction_lag_jacobian(S, kind, xs, eps_x):
    """The lagged friction data of one pair at x_t (Eq. 3, E_friction) and their derivatives with respect
    to the pair's four positions at x_t (12 columns).

    lambda = -kappa m 2 d b'(s) (s = d^2 the squared distance, m the edge-edge mollifier); n = v / d with
    v = sum_q w_q x_q the vector between the closest points; w the closest-point weights.  Within one
    distance type the weights minimise |V w|^2 over w = w0 + B theta (V the 3x4 matrix of positions), so
    with A = V B the optimality condition A^T v = 0 gives, for a change dV,
    d theta = -(A^T A)^-1 (dA^T v + A^T dV w)."""
    xs = _f64(xs).reshape(4, 3)
    t, s, w = classify(kind, xs)
    _, gs, _ = (pt_dist if kind == 0 else ee_dist)(xs, t)
    d = math.sqrt(s)
    v = (w[:, None] * xs).sum(0)
    n = v / d
    _, b1, b2 = barrier(s, S.sh)
    if kind == 1:
        m, gm, _ = ee_mollifier(xs, eps_x)
    else:
        m, gm = 1.0, np.zeros(12)
    lam = -S.kappa * m * 2.0 * d * b1
    dlam = -S.kappa * (2.0 * d * b1 * gm + m * (b1 / d + 2.0 * d * b2) * gs)
    B = _free_weight_directions(kind, t)
    dw = np.zeros((4, 12))
    if B.shape[1]:
        A = xs.T @ B
        G = A.T @ A
        for j in range(4):
            for dd in range(3):
                rhs = B[j, :] * v[dd] + A[dd, :] * w[j]
                dw[:, 3 * j + dd] = B @ (-np.linalg.solve(G, rhs))
    dv = np.zeros((3, 12))
    for j in range(4):
        for dd in range(3):
            dv[dd, 3 * j + dd] += w[j]
    dv += xs.T @ dw
    dn = (np.eye(3) - np.outer(n, n)) @ dv / d
    return dict(type=t, w=w, n=n, lam=lam, dw=dw, dn=dn, dlam=dlam)


def friction_lag_adjoint(S, ctx, x, lv):
    """The part of dL/dx_t that flows through the lagged friction data (lambda_k, n_k, w_k at x_t), in
    vertex space, for the vertex-space adjoint lv of one step.  Per pair
    Phi = lv . grad_x D = mu lambda phi(r) a^T y,  a = sum_q w_q lv_q,  y = (I - n n^T) u,
    u = sum_q w_q (x_q - x_t,q),  r = |y|,  phi(r) = f0'(r) / r,
    and the contribution is -dt^2 dPhi/dx_t through lambda, n and w (the direct dependence of u on x_t is
    the friction Hessian term of the adjoint)."""
    out = np.zeros((S.nv, 3))
    xt = ctx["x_t"]
    eps = S.eps
    for (ids, w0, n0, lam0), kind, eps_x in zip(ctx["lag"], ctx["lag_kind"], ctx["lag_eps_x"]):
        J = friction_lag_jacobian(S, kind, xt[ids], eps_x)
        w, n, lam = J["w"], J["n"], J["lam"]
        u = (w[:, None] * (x[ids] - xt[ids])).sum(0)
        T = np.eye(3) - np.outer(n, n)
        y = T @ u
        r = math.sqrt(float(y @ y))
        phi = (-r / (eps * eps) + 2.0 / eps) if r < eps else 1.0 / r
        dphi_over_r = ((-1.0 / (eps * eps)) / r if r > 0 else 0.0) if r < eps else -1.0 / (r ** 3)
        a = (w[:, None] * lv[ids]).sum(0)
        c2 = S.mu_f * lam * phi
        c1 = S.mu_f * lam * dphi_over_r * float(a @ y)
        Phi = c2 * float(a @ y)
        z = c1 * y + c2 * a
        g_u = c1 * y + c2 * (T @ a)
        g_n = -(z * float(n @ u) + u * float(n @ z))
        dPhi_dw = np.array([c2 * float(y @ lv[ids[q]]) + float(g_u @ (x[ids[q]] - xt[ids[q]])) for q in range(4)])
        grad = (Phi / lam) * J["dlam"] + g_n @ J["dn"] + dPhi_dw @ J["dw"]
        np.add.at(out, ids, -S.dt * S.dt * grad.reshape(4, 3))
    return out


def adjoint_step(o: "Oracle", z_t, zd_t, z_next, step_next, gz_next, gzd_next):
    """Backward of one step by the implicit function theorem.

    At the converged z* the free-DOF gradient g(z*; z_t, zd_t, theta) vanishes,
    so with H = dg/dz (the unprojected Hessian, dense here) and
    a = dL/dz* + dL/dzd* / dt (zd* = (z* - z_t) / dt):
        H lam = a,  dL/dtheta = -lam^T dg/dtheta,
        dL/dz_t = M lam - dL/dzd* / dt + dt^2 H_fric lam,   dL/dzd_t = dt M lam.
    theta = per-tet log E: dg/dlogE_e = dt^2 (gradient of V_e Psi_e), since
    Psi is linear in (mu, lam) and both scale with E; dg/dmu = dt^2 grad D / mu.
    The friction lag (lambda_k, n_k, w_k computed at x_t) depends on x_t too;
    that dependence is differentiated by friction_lag_adjoint.
    Returns (dL/dz_t, dL/dzd_t, dL/dlogE, dL/dmu) on the free DOFs."""
    S = o.S
    dt = S.dt
    F = slice(0, S.n_free)
    ctx = step_context(S, z_t, zd_t, step_next)
    _, _, H, _ = S.evaluate(z_next, ctx, project=False)
    HFF = H.tocsr()[F, F].toarray()
    a = (gz_next + gzd_next / dt)[F]
    lam = np.linalg.solve(HFF, a)
    lam_full = np.zeros(S.ndof)
    lam_full[F] = lam
    # theta = log E per tet
    x = S.positions(z_next).reshape(-1)
    dlogE = np.zeros(len(S.tets))
    lv = (S.Jmap @ lam_full).reshape(-1, 3)
    for e in range(len(S.tets)):
        ids = S.tets[e]
        _, ge, _ = tet(x.reshape(-1, 3)[ids], S.B[e], S.vol[e], S.mu[e], S.lam[e])
        dlogE[e] = -dt * dt * float(ge @ lv[ids].reshape(-1))
    # friction coefficient and the direct x_t dependence of the friction term
    dmu = 0.0
    fr_rows, fr_cols, fr_vals = [], [], []
    xt = ctx["x_t"]
    for ids, w, nvec, lamk in ctx["lag"]:
        Ek, gk, Hk = friction(w, nvec, lamk, S.mu_f, S.eps, x.reshape(-1, 3)[ids], xt[ids])
        dmu += -dt * dt * float(gk @ lv[ids].reshape(-1)) / S.mu_f
        dofs = (3 * ids[:, None] + np.arange(3)).reshape(-1)
        fr_rows.append(np.repeat(dofs, 12)); fr_cols.append(np.tile(dofs, 12)); fr_vals.append(Hk.reshape(-1))
    gz_t = S.M @ lam_full - gzd_next / dt
    if fr_vals:
        import scipy.sparse as sp
        Hf = sp.csr_matrix((np.concatenate(fr_vals), (np.concatenate(fr_rows), np.concatenate(fr_cols))),
                           shape=(3 * S.nv, 3 * S.nv))
        gz_t = gz_t + dt * dt * (S.Jmap.T @ (Hf @ (S.Jmap @ lam_full)))
        gz_t = gz_t + S.Jmap.T @ friction_lag_adjoint(S, ctx, x.reshape(-1, 3), lv).reshape(-1)
    gzd_t = dt * (S.M @ lam_full)
    gz_t[S.n_free:] = 0.0
    gzd_t[S.n_free:] = 0.0
    return gz_t, gzd_t, dlogE, dmu
