"""Seeded synthetic scene generators (inputs only).

This module produces the geometry, materials, kinematic trajectories and
parameters of the grasp scenes that the IPC step (Eq. 3, §III-C.2) is run on.
It holds none of the method's arithmetic: no surface extraction, no rest
shape matrices, no masses, no energies.  Both the CUDA path and the CPU
oracle consume the dictionaries it returns.

Random numbers come from splitmix64 (Steele, Lea, Flood 2014), written out
here from its published definition so any consumer can regenerate them.

Units are SI (metres, seconds, kilograms, pascals).

A scene dictionary has the keys

  fem_X      (nv, 3) float64  rest = initial positions of all FEM vertices
  fem_tets   (nt, 4) int32    tetrahedra, positively oriented
  fem_logE   (nt,)   float64  natural log of Young's modulus per tet
  fem_nu     (nt,)   float64  Poisson ratio per tet
  fem_rho    (nt,)   float64  density per tet
  fem_body   (nt,)   int32    FEM body id per tet (fingertip 0, 1, object ...)
  kin        list of {"X": (n,3) local rest vertices, "tris": (m,3) int32}
  kin_T      (n_steps + 1, n_kin, 3, 4) rigid transforms [R | t] per step
  abd        list of {"X": (n,3) body-frame vertices, "tris": (m,3) int32,
                      "rho": float, "q0": (12,) [p, A[:,0], A[:,1], A[:,2]]}
  stitch_v   (ns,) int32      FEM vertex of each stitch spring (Eq. 2)
  stitch_b   (ns,) int32      kinematic body carrying the anchor
  stitch_X   (ns, 3) float64  anchor point in that body's local frame
  gravity    (3,) float64
  params     dict of scalar parameters (see ``default_params``)
"""
from __future__ import annotations

import math
import numpy as np

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64: state += golden gamma, then two xor-shift-multiply rounds."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1): top 53 bits of each draw times 2^-53."""
        out = np.empty(n, dtype=np.float64)
        for i in range(n):
            out[i] = (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)
        return out

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by Box-Muller on pairs of uniforms."""
        m = (n + 1) // 2
        u = self.uniform(2 * m)
        u1 = 1.0 - u[0::2]
        u2 = u[1::2]
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return z[:n]


def default_params(**kw) -> dict:
    p = dict(
        dt=1e-2,          # time step (s)
        dhat=1e-3,        # barrier activation distance (m)
        kappa=0.0,        # barrier stiffness; 0 = auto-scaled at create
        mu=0.5,           # friction coefficient
        eps_v=1e-3,       # friction static-velocity threshold (m/s)
        k_c=0.0,          # stitch stiffness (N/m); 0 = auto
        kappa_A=1e8,      # ABD orthogonality stiffness (Pa)
        newton_tol=1e-6,  # ||p||_inf / (dt * L_bbox)
        pcg_rtol=1e-4,
        max_newton=100,
        max_pcg=0,        # 0 = 10 * sqrt(n_dof)
        s_ccd=0.1,        # ACCD minimum-separation fraction
        n_steps=20,
    )
    p.update(kw)
    return p


# ----------------------------------------------------------------------------
# mesh builders
# ----------------------------------------------------------------------------

def grid_tets(origin, cell, nx, ny, nz):
    """Regular grid of cubes, each cut into 6 tets around its main diagonal.

    The split follows the Kuhn (Freudenthal) scheme: every cube uses the same
    diagonal from corner (0,0,0) to (1,1,1), which makes the mesh conforming.
    Returns (verts (nv,3), tets (nt,4) int32), tets positively oriented.
    """
    ox, oy, oz = origin
    hx, hy, hz = cell if np.ndim(cell) else (cell, cell, cell)
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    verts = np.stack([ox + ii * hx, oy + jj * hy, oz + kk * hz], axis=-1)
    verts = verts.transpose(2, 1, 0, 3).reshape(-1, 3)  # index = i + (nx+1)(j + (ny+1)k)

    def vid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    perms = [(0, 1, 2, +1), (1, 2, 0, +1), (2, 0, 1, +1), (0, 2, 1, -1), (2, 1, 0, -1), (1, 0, 2, -1)]
    tets = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for a0, a1, a2, sgn in perms:
                    c0 = [0, 0, 0]
                    c1 = list(c0); c1[a0] = 1
                    c2 = list(c1); c2[a1] = 1
                    c3 = [1, 1, 1]
                    v = [vid(i + c[0], j + c[1], k + c[2]) for c in (c0, c1, c2, c3)]
                    if sgn < 0:
                        v[1], v[2] = v[2], v[1]
                    tets.append(v)
    return verts.astype(np.float64), np.asarray(tets, dtype=np.int32)


def box_surface(lo, hi):
    """Closed box surface: 8 verts, 12 outward-facing triangles."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    v = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float64)
    t = np.array([[0, 2, 1], [0, 3, 2],   # bottom (-z)
                  [4, 5, 6], [4, 6, 7],   # top (+z)
                  [0, 1, 5], [0, 5, 4],   # -y
                  [2, 3, 7], [2, 7, 6],   # +y
                  [1, 2, 6], [1, 6, 5],   # +x
                  [3, 0, 4], [3, 4, 7]],  # -x
                 dtype=np.int32)
    return v, t


def uv_ellipsoid(a, b, c, n_lat, n_lon):
    """Closed ellipsoid surface, outward triangles, 2 + (n_lat-1) n_lon verts."""
    verts = [[0.0, 0.0, c]]
    for i in range(1, n_lat):
        th = math.pi * i / n_lat
        for j in range(n_lon):
            ph = 2 * math.pi * j / n_lon
            verts.append([a * math.sin(th) * math.cos(ph), b * math.sin(th) * math.sin(ph), c * math.cos(th)])
    verts.append([0.0, 0.0, -c])
    tris = []
    for j in range(n_lon):
        tris.append([0, 1 + j, 1 + (j + 1) % n_lon])
    for i in range(n_lat - 2):
        r0 = 1 + i * n_lon
        r1 = r0 + n_lon
        for j in range(n_lon):
            j1 = (j + 1) % n_lon
            tris.append([r0 + j, r1 + j, r1 + j1])
            tris.append([r0 + j, r1 + j1, r0 + j1])
    last = len(verts) - 1
    r0 = 1 + (n_lat - 2) * n_lon
    for j in range(n_lon):
        tris.append([last, r0 + (j + 1) % n_lon, r0 + j])
    return np.asarray(verts, dtype=np.float64), np.asarray(tris, dtype=np.int32)


def superellipsoid_capsule(rx, ry, length, n_ring, n_seg, expo=2.5):
    """Convex-ish link shell: super-elliptic cross-section swept along z, hemispherical-ish caps."""
    verts = []
    n_cap = max(2, n_ring // 4)
    rings = []
    for i in range(n_cap, 0, -1):  # bottom cap
        th = 0.5 * math.pi * i / (n_cap + 1)
        rings.append((math.cos(th), -math.sin(th) * min(rx, ry)))
    for i in range(n_seg + 1):
        rings.append((1.0, length * i / n_seg))
    for i in range(1, n_cap + 1):  # top cap
        th = 0.5 * math.pi * i / (n_cap + 1)
        rings.append((math.cos(th), length + math.sin(th) * min(rx, ry)))
    verts.append([0.0, 0.0, -min(rx, ry)])
    for scale, z in rings:
        for j in range(n_ring):
            ph = 2 * math.pi * j / n_ring
            c, s = math.cos(ph), math.sin(ph)
            e = 2.0 / expo
            x = rx * scale * math.copysign(abs(c) ** e, c)
            y = ry * scale * math.copysign(abs(s) ** e, s)
            verts.append([x, y, z])
    verts.append([0.0, 0.0, length + min(rx, ry)])
    nr = len(rings)
    tris = []
    for j in range(n_ring):
        tris.append([0, 1 + (j + 1) % n_ring, 1 + j])
    for i in range(nr - 1):
        r0 = 1 + i * n_ring
        r1 = r0 + n_ring
        for j in range(n_ring):
            j1 = (j + 1) % n_ring
            tris.append([r0 + j, r0 + j1, r1 + j1])
            tris.append([r0 + j, r1 + j1, r1 + j])
    last = len(verts) - 1
    r0 = 1 + (nr - 1) * n_ring
    for j in range(n_ring):
        tris.append([last, r0 + j, r0 + (j + 1) % n_ring])
    return np.asarray(verts, dtype=np.float64), np.asarray(tris, dtype=np.int32)


def translation(t):
    T = np.zeros((3, 4))
    T[:, :3] = np.eye(3)
    T[:, 3] = t
    return T


def rot_z(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1.0]])


def rot_y(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])


def rot_x(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])


def _empty_stitch():
    return (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros((0, 3)))


# ----------------------------------------------------------------------------
# workload 1: one soft fingertip pressed by a plate onto a fixed cube
# ----------------------------------------------------------------------------

def fingertip_press(seed: int = 0, n_steps: int = 20, **param_overrides) -> dict:
    """10 x 6 x 20 mm soft box (5 x 3 x 10 cubes, 6 tets each: 264 verts, 900 tets).

    E = 1e5 Pa, nu = 0.45, rho = 1100 kg/m^3.  The box stands 0.5 mm above a
    fixed 30 mm rigid cube (top face at z = 0).  A 30 x 30 x 2 mm kinematic
    plate starts 0.5 mm above the box top and moves down 0.1 mm per step
    (2 mm over 20 steps).  Every rest coordinate gets uniform +/- 0.1 mm
    jitter from splitmix64(seed); rest = initial, so the box starts unstressed.
    """
    mm = 1e-3
    X, tets = grid_tets((-5 * mm, -3 * mm, 0.5 * mm), 2 * mm, 5, 3, 10)
    rng = SplitMix64(seed)
    X = X + (2.0 * rng.uniform(X.size).reshape(X.shape) - 1.0) * 0.1 * mm
    nt = tets.shape[0]
    cube_X, cube_T = box_surface((-15 * mm, -15 * mm, -30 * mm), (15 * mm, 15 * mm, 0.0))
    plate_X, plate_T = box_surface((-15 * mm, -15 * mm, 0.0), (15 * mm, 15 * mm, 2 * mm))
    kin_T = np.zeros((n_steps + 1, 2, 3, 4))
    for s in range(n_steps + 1):
        kin_T[s, 0] = translation((0.0, 0.0, 0.0))
        kin_T[s, 1] = translation((0.0, 0.0, 21 * mm - 0.1 * mm * s))
    sv, sb, sx = _empty_stitch()
    params = default_params(dt=1e-2, dhat=1e-3, mu=0.5, newton_tol=1e-6, n_steps=n_steps)
    params.update(param_overrides)
    return dict(
        name="fingertip_press_900tet",
        fem_X=X, fem_tets=tets,
        fem_logE=np.full(nt, math.log(1e5)), fem_nu=np.full(nt, 0.45), fem_rho=np.full(nt, 1100.0),
        fem_body=np.zeros(nt, np.int32),
        kin=[dict(X=cube_X, tris=cube_T), dict(X=plate_X, tris=plate_T)],
        kin_T=kin_T,
        abd=[],
        stitch_v=sv, stitch_b=sb, stitch_X=sx,
        gravity=np.array([0.0, 0.0, -9.81]),
        params=params,
    )


def free_block(n_steps: int = 5, v0=(0.0, 0.0, 0.0), **param_overrides) -> dict:
    """A 2 x 2 x 2 mm single-cube block (6 tets) with no obstacles: free fall."""
    mm = 1e-3
    X, tets = grid_tets((0.0, 0.0, 0.0), 2 * mm, 1, 1, 1)
    nt = tets.shape[0]
    sv, sb, sx = _empty_stitch()
    params = default_params(n_steps=n_steps)
    params.update(param_overrides)
    sc = dict(
        name="free_block",
        fem_X=X, fem_tets=tets,
        fem_logE=np.full(nt, math.log(1e5)), fem_nu=np.full(nt, 0.45), fem_rho=np.full(nt, 1100.0),
        fem_body=np.zeros(nt, np.int32),
        kin=[], kin_T=np.zeros((n_steps + 1, 0, 3, 4)), abd=[],
        stitch_v=sv, stitch_b=sb, stitch_X=sx,
        gravity=np.array([0.0, 0.0, -9.81]),
        params=params,
    )
    sc["fem_V0"] = np.tile(np.asarray(v0, dtype=np.float64), (X.shape[0], 1))
    return sc


def block_on_plane(n_steps: int = 10, tilt: float = 0.0, mu: float = 0.5, **param_overrides) -> dict:
    """4 x 4 x 4 mm block (4^3 cubes of 1 mm) starting 0.3 mm above a fixed plane tilted by `tilt` about y."""
    mm = 1e-3
    X, tets = grid_tets((-2 * mm, -2 * mm, 0.3 * mm), 1 * mm, 4, 4, 4)
    nt = tets.shape[0]
    # one large ground triangle whose edges are all far from the block
    gX = np.array([[-50 * mm, -50 * mm, 0.0], [250 * mm, -50 * mm, 0.0], [-50 * mm, 250 * mm, 0.0]])
    gT = np.array([[0, 1, 2]], dtype=np.int32)
    R = rot_y(tilt)
    X = X @ R.T
    kin_T = np.zeros((n_steps + 1, 1, 3, 4))
    for s in range(n_steps + 1):
        kin_T[s, 0, :, :3] = R
    sv, sb, sx = _empty_stitch()
    params = default_params(dt=1e-2, dhat=2e-4, mu=mu, n_steps=n_steps)
    params.update(param_overrides)
    return dict(
        name="block_on_plane",
        fem_X=X, fem_tets=tets,
        fem_logE=np.full(nt, math.log(1e5)), fem_nu=np.full(nt, 0.4), fem_rho=np.full(nt, 1000.0),
        fem_body=np.zeros(nt, np.int32),
        kin=[dict(X=gX, tris=gT)], kin_T=kin_T, abd=[],
        stitch_v=sv, stitch_b=sb, stitch_X=sx,
        gravity=np.array([0.0, 0.0, -9.81]),
        params=params,
    )


# ----------------------------------------------------------------------------
# workload 2: arm-gripper grasp of a rigid ellipsoid (FP64)
# ----------------------------------------------------------------------------

def subdivided_box(lo, hi, n):
    """Closed box surface with every face cut into n x n quads (2 n^2 triangles per face), outward."""
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    verts = {}
    vlist = []

    def vid(p):
        key = tuple(np.round(p, 12))
        if key not in verts:
            verts[key] = len(vlist)
            vlist.append(p)
        return verts[key]

    tris = []
    for axis in range(3):
        for side in (0, 1):
            a1, a2 = [a for a in range(3) if a != axis]
            for i in range(n):
                for j in range(n):
                    def P(ii, jj):
                        p = np.zeros(3)
                        p[axis] = hi[axis] if side else lo[axis]
                        p[a1] = lo[a1] + (hi[a1] - lo[a1]) * ii / n
                        p[a2] = lo[a2] + (hi[a2] - lo[a2]) * jj / n
                        return vid(p)
                    q = [P(i, j), P(i + 1, j), P(i + 1, j + 1), P(i, j + 1)]
                    # outward: (a1 x a2) points along +axis for cyclic (axis, a1, a2)
                    cyclic = (a1 - axis) % 3 == 1
                    flip = (side == 0) == cyclic
                    if flip:
                        tris.append([q[0], q[2], q[1]]); tris.append([q[0], q[3], q[2]])
                    else:
                        tris.append([q[0], q[1], q[2]]); tris.append([q[0], q[2], q[3]])
    return np.asarray(vlist, dtype=np.float64), np.asarray(tris, dtype=np.int32)


def morton_order(X, T):
    """The mesh (X, T) with its vertices renumbered in Morton (Z-curve) order of their positions, so that
    consecutive vertex ids are spatially close (the usual reordering of a generated tet mesh: runs of
    consecutive vertices form compact clusters)."""
    lo = X.min(0)
    ext = float((X.max(0) - lo).max()) or 1.0
    q = np.floor((X - lo) / ext * 1023.0).astype(np.int64)
    code = np.zeros(len(X), np.int64)
    for bit in range(10):
        for d in range(3):
            code |= ((q[:, d] >> bit) & 1) << (3 * bit + d)
    order = np.argsort(code, kind="stable")
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    return X[order], inv[T].astype(np.int32)


def finray_tip(h=1.25e-3, width=20e-3, height=40e-3, depth=20e-3):
    """Voxelised fin-ray fingertip in its local frame (u, v, w).

    Profile: the right triangle u in [0, width], w in [0, height],
    u / width + w / height <= 1 (contact face u = 0, mounting face w = 0, back
    face the hypotenuse), extruded over v in [0, depth].  Three slanted rib
    voids (one cell thick) run between the contact face and the back face.
    Cells are cut into 6 tets each; vertices are numbered in Morton order."""
    nu, nw, nv = int(round(width / h)), int(round(height / h)), int(round(depth / h))
    keep = np.zeros((nu, nv, nw), bool)
    for i in range(nu):
        for k in range(nw):
            uc, wc = (i + 0.5) * h, (k + 0.5) * h
            if uc / width + wc / height > 1.0:
                continue
            keep[i, :, k] = True
            # rib voids: bands along w = w0 + 0.6 u, away from the outer walls
            umax = width * (1.0 - wc / height)
            for w0 in (0.25 * height, 0.45 * height, 0.65 * height):
                if abs(wc - (w0 + 0.6 * uc)) < 0.5 * h and 2 * h < uc < umax - 2 * h:
                    keep[i, 1:nv - 1, k] = False
    X, T = grid_tets((0.0, 0.0, 0.0), h, nu, nv, nw)
    cell_of_tet = np.repeat(np.arange(nu * nv * nw), 6)
    # grid_tets enumerates cells k-major, then j, then i
    ci = np.arange(nu * nv * nw)
    ii = ci % nu
    jj = (ci // nu) % nv
    kk = ci // (nu * nv)
    cell_keep = keep[ii, jj, kk]
    T = T[cell_keep[cell_of_tet]]
    used = np.unique(T)
    remap = -np.ones(len(X), np.int64)
    remap[used] = np.arange(len(used))
    return morton_order(X[used], remap[T].astype(np.int32))


def _frame(R, t):
    T = np.zeros((3, 4))
    T[:, :3] = R
    T[:, 3] = t
    return T


def arm_gripper_grasp(seed: int = 0, n_steps: int = 400, tip_cell=1.25e-3, link_tris=2000, obj_tris=5000,
                      base_tris=1000, close_per_step=0.05e-3, close_steps=100, hold_steps=20, lift_per_step=0.25e-3,
                      **param_overrides) -> dict:
    """Two fin-ray fingertips (E = 2e5 Pa, nu = 0.45, rho = 1100) stitched to
    two kinematic finger bases grasp and lift a rigid ABD ellipsoid (semi-axes
    30/25/20 mm, 0.1 kg) resting on a kinematic ground quad; seven kinematic
    arm links (~2k triangles each) follow the gripper with seeded smooth
    joint wobble.  dt = 5 ms, dhat = 0.5 mm, mu = 0.6.

    Trajectory: the fingertips start in the pre-grasp pose 0.8 mm from the
    object, close 0.05 mm per step for 100 steps (5 mm), hold 20 steps, then
    the gripper and arm lift at 50 mm/s (0.25 mm per step).  The resolution
    (tip voxel size, link, object and base triangle counts) and the
    trajectory timing are parameters, so that a reduced scene with every
    ingredient fits the CPU oracle."""
    mm = 1e-3
    rng = SplitMix64(seed)
    a, b, c = 30 * mm, 25 * mm, 20 * mm
    # object
    n_lon = max(8, int(round(math.sqrt(obj_tris * 1.6 / 2))))
    n_lat = max(4, int(round(obj_tris / (2 * n_lon))) + 1)
    oX, oT = uv_ellipsoid(a, b, c, n_lat, n_lon)
    vol = 4.0 / 3.0 * math.pi * a * b * c
    rho_obj = 0.1 / vol
    q0 = np.concatenate([[0.0, 0.0, c + 0.3 * mm], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    # fingertips (local u: away from the object, v: along x, w: down)
    tX, tT = finray_tip(h=tip_cell)
    height = 40 * mm
    z_top = q0[2] + 22 * mm
    gap = 0.8 * mm
    Xs, Ts = [], []
    fem_body = []
    offs = 0
    tips = []
    for side in (+1, -1):
        # world = (x: v - depth/2, y: side * (b + gap + u), z: z_top - w)
        Xw = np.stack([tX[:, 1] - 10 * mm, side * (b + gap + tX[:, 0]), z_top - tX[:, 2]], axis=1)
        T = tT.copy()
        if side < 0:
            T[:, [1, 2]] = T[:, [2, 1]]  # the mirror flips orientation
        Xs.append(Xw)
        Ts.append(T + offs)
        fem_body.append(np.full(len(T), len(tips), np.int32))
        tips.append((offs, len(Xw)))
        offs += len(Xw)
    X = np.concatenate(Xs)
    tets = np.concatenate(Ts)
    fem_body = np.concatenate(fem_body)
    nt = len(tets)
    # finger bases: kinematic boxes 0.6 mm above each tip's mounting face (~1k triangles)
    base_n = max(1, int(round(math.sqrt(base_tris / 12))))
    kin = []
    base_up, base_tris = subdivided_box((-12 * mm, -2 * mm, 0.6 * mm), (12 * mm, 22 * mm, 8.6 * mm), base_n)
    base_dn = base_up * np.array([1.0, -1.0, 1.0])  # mirror image for the -y finger
    # ground quad, diagonal well away from the object
    g = 0.5
    gX = np.array([[-g + 0.2, -g + 0.3, 0], [g + 0.2, -g + 0.3, 0], [g + 0.2, g + 0.3, 0], [-g + 0.2, g + 0.3, 0.0]])
    gT = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    kin.append(dict(X=gX, tris=gT))                   # body 0: ground
    kin.append(dict(X=base_up, tris=base_tris))                        # body 1: base of tip +y
    kin.append(dict(X=base_dn, tris=base_tris[:, [0, 2, 1]].copy()))   # body 2: base of tip -y
    # arm links: capsules above the gripper, ~link_tris triangles each
    n_ring = max(8, int(round(math.sqrt(link_tris / 2))))
    n_seg = max(2, int(round(link_tris / (2 * n_ring))) - n_ring // 2)
    links = []
    for k in range(7):
        lX, lT = superellipsoid_capsule(28 * mm - 2 * mm * k, 24 * mm - 2 * mm * k, 60 * mm, n_ring, n_seg)
        kin.append(dict(X=lX, tris=lT))
        links.append(k)
    # stitch springs: tip vertices on the mounting face (w <= 0.5 mm) to their base
    sv, sb, sx = [], [], []
    for ti, side in enumerate((+1, -1)):
        o, n = tips[ti]
        for v in range(o, o + n):
            if z_top - X[v, 2] <= 0.5 * mm:
                sv.append(v)
                sb.append(1 + ti)
                # anchor in the base frame (axis-aligned, origin (0, side (b + gap), z_top))
                sx.append([X[v, 0], X[v, 1] - side * (b + gap), X[v, 2] - z_top])
    # trajectory
    phases = np.zeros(n_steps + 1)
    lift = np.zeros(n_steps + 1)
    for s in range(n_steps + 1):
        phases[s] = min(s, close_steps) * close_per_step
        lift[s] = max(0, s - close_steps - hold_steps) * lift_per_step
    wob_amp = 0.02 * rng.uniform(7)
    wob_w = 2 * math.pi * (0.5 + rng.uniform(7))
    wob_ph = 2 * math.pi * rng.uniform(7)
    dt = 5e-3
    kin_T = np.zeros((n_steps + 1, len(kin), 3, 4))
    for s in range(n_steps + 1):
        kin_T[s, 0] = _frame(np.eye(3), (0, 0, 0))
        for ti, side in enumerate((+1, -1)):
            y0 = side * (b + gap - phases[s])
            kin_T[s, 1 + ti] = _frame(np.eye(3), (0.0, y0, z_top + lift[s]))
        t = s * dt
        for k in range(7):
            ang = wob_amp[k] * math.sin(wob_w[k] * t + wob_ph[k])
            R = rot_z(ang + 0.3 * k) @ rot_x(0.05 * k)
            kin_T[s, 3 + k] = _frame(R, (0.0, 0.0, z_top + 40 * mm + 75 * mm * k + lift[s]))
    params = default_params(dt=dt, dhat=0.5 * mm, mu=0.6, newton_tol=1e-6, n_steps=n_steps)
    params.update(param_overrides)
    return dict(
        name=f"arm_gripper_grasp_{nt}tet",
        fem_X=X, fem_tets=tets,
        fem_logE=np.full(nt, math.log(2e5)), fem_nu=np.full(nt, 0.45), fem_rho=np.full(nt, 1100.0),
        fem_body=fem_body,
        kin=kin, kin_T=kin_T,
        abd=[dict(X=oX, tris=oT, rho=rho_obj, q0=q0)],
        stitch_v=np.asarray(sv, np.int32), stitch_b=np.asarray(sb, np.int32), stitch_X=np.asarray(sx, np.float64),
        gravity=np.array([0.0, 0.0, -9.81]),
        params=params,
    )


def arm_gripper_grasp_reduced(seed: int = 0, n_steps: int = 16, **param_overrides) -> dict:
    """Every ingredient of the arm-gripper grasp at a resolution the CPU oracle
    steps in seconds: two fin-ray tips of 3 mm voxels (about 1.8k tets each), 7 kinematic arm links
    of about 50 triangles on the seeded joint wobble, two stitched finger bases
    of about 100 triangles, the ABD ellipsoid (about 300 triangles, 0.1 kg) on
    the ground quad, mu = 0.6.  Faster trajectory: contact at about step 3,
    squeeze to step 10 (0.3 mm per step), hold 2 steps, then lift."""
    sc = arm_gripper_grasp(seed, n_steps=n_steps, tip_cell=3.0e-3, link_tris=48, obj_tris=300, base_tris=100,
                           close_per_step=0.3e-3, close_steps=10, hold_steps=2, **param_overrides)
    sc["name"] = f"arm_gripper_grasp_reduced_{len(sc['fem_tets'])}tet"
    return sc


def material_identification(seed: int = 0, n_steps: int = 100, tip_cell=0.97e-3, hidden_seed: int = 1,
                            sigma: float = 0.3, **param_overrides) -> dict:
    """Differentiable material identification: the arm-gripper grasp refined to about 100k tets (two
    fin-ray tips of 0.97 mm voxels) with per-tet ln Young's modulus drawn lognormal around 2e5 Pa
    (sigma 0.3, seed `seed`) as the parameters to identify, mu = 0.6.  The returned scene also holds the
    hidden parameters (`hidden_logE`, seed `hidden_seed`, and `hidden_mu` = 0.5) that simulate the target
    trajectory of the loss."""
    sc = arm_gripper_grasp(0, n_steps=n_steps, tip_cell=tip_cell, **param_overrides)
    nt = len(sc["fem_tets"])
    sc["fem_logE"] = math.log(2e5) + sigma * SplitMix64(seed + 7000).normal(nt)
    sc["hidden_logE"] = math.log(2e5) + sigma * SplitMix64(hidden_seed + 7000).normal(nt)
    sc["hidden_mu"] = 0.5
    sc["name"] = f"material_identification_{nt}tet"
    return sc


def render_setup(sc: dict, sim_surface_tris, n_sim_verts: int, seed: int = 0):
    """A render scene around a simulation scene: the simulated surface triangles (global vertex ids) as
    diffuse surfaces (fingertips light grey, affine bodies orange, kinematic bodies dark grey), a
    reconstructed-background stand-in (a 1.2 m table top and a back wall cut into quads with a seeded
    per-quad texture colour, Eq. 7 material), two rectangular area lights, and a camera looking at the
    gripper.  Returns (extra vertices (m, 3) appended after the simulated ones, triangles, material per
    triangle, colour per triangle, camera (13 floats, width, height))."""
    rng = SplitMix64(seed + 9000)
    nf = len(sc["fem_X"])
    n_abd_v = sum(a["X"].shape[0] for a in sc.get("abd", []))
    tris = [np.asarray(sim_surface_tris, np.int64)]
    t = tris[0]
    kind = np.where(t.max(1) < nf, 0, np.where(t.max(1) < nf + n_abd_v, 1, 2))
    rgb = [np.array([[0.75, 0.75, 0.72], [0.9, 0.5, 0.15], [0.25, 0.25, 0.28]])[kind]]
    types = [np.zeros(len(t), np.int64)]
    extra = []
    base = n_sim_verts

    def add_quad(c, u, v, mtype, colour):
        nonlocal base
        c, u, v = (np.asarray(a, float) for a in (c, u, v))
        extra.append(np.array([c - u - v, c + u - v, c + u + v, c - u + v]))
        tris.append(np.array([[base, base + 1, base + 2], [base, base + 2, base + 3]]))
        types.append(np.full(2, mtype))
        rgb.append(np.tile(np.asarray(colour, float), (2, 1)))
        base += 4

    cells = 12
    half = 0.6 / cells
    u = rng.uniform(3 * 2 * cells * cells)
    k = 0
    for i in range(cells):
        for j in range(cells):
            # table top: warm wood-like noise; back wall: cool grey noise
            add_quad((-0.6 + (2 * i + 1) * half, -0.6 + (2 * j + 1) * half, -1e-4), (half, 0, 0), (0, half, 0), 2,
                     0.45 + 0.25 * u[3 * k:3 * k + 3] * np.array([1.0, 0.8, 0.5]))
            k += 1
            add_quad((-0.6 + (2 * i + 1) * half, 0.3, (2 * j + 1) * half), (half, 0, 0), (0, 0, half), 2,
                     0.55 + 0.2 * u[3 * k:3 * k + 3] * np.array([0.8, 0.85, 1.0]))
            k += 1
    add_quad((-0.15, -0.1, 0.45), (0.08, 0, 0), (0, 0.08, 0), 1, [12.0, 11.5, 10.5])
    add_quad((0.2, -0.25, 0.35), (0.05, 0, 0), (0, 0, 0.05), 1, [6.0, 6.5, 7.0])
    eye = np.array([0.0, -0.32, 0.16])
    target = np.array([0.0, 0.0, 0.05])
    f = (target - eye) / np.linalg.norm(target - eye)
    r = np.cross(f, [0, 0, 1.0]); r /= np.linalg.norm(r)
    up = np.cross(r, f)
    cam = (np.concatenate([eye, f, r, up, [math.tan(math.radians(45.0) / 2)]]).astype(np.float32), 640, 360)
    return (np.concatenate(extra), np.concatenate(tris).astype(np.int32), np.concatenate(types).astype(np.int32),
            np.concatenate(rgb).astype(np.float32), cam)


def jointed_arm(n_links: int = 3, n_steps: int = 12, swing: float = 0.6, with_block: bool = True,
                gravity: bool = True, **param_overrides) -> dict:
    """A planar arm of affine (ABD) links joined by revolute joints with drive potentials (E_joint of
    Eq. 3): link i is a 40 x 8 x 8 mm box (density 1000), hinged to link i - 1 (link 0 to the world) about
    the vertical axis by two point springs on the hinge axis (k 2e4 N/m; the boxes stop 4 mm short of
    the hinges, so that neighbouring links stay apart when they turn), and driven toward its joint angle
    theta_i(t) by a direction spring between the link's axis and the parent's axis turned by theta_i
    (k 40 N/m).  The joint angles ramp to `swing` (rad, sign alternating) over the first steps, sweeping
    the tip into a soft 10 mm block (E 1e5) resting on a ground triangle.  Scene keys joints / joint_b /
    joint_t describe the joints and their per-step drive targets."""
    mm = 1e-3
    L, w, gap = 40 * mm, 8 * mm, 4 * mm
    lX, lT = subdivided_box((-L / 2 + gap, -w / 2, -w / 2), (L / 2 - gap, w / 2, w / 2), 2)
    z0 = 12 * mm
    abd, joints = [], []
    for i in range(n_links):
        q0 = np.concatenate([[L * i + L / 2, 0.0, z0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
        abd.append(dict(X=lX.copy(), tris=lT.copy(), rho=1000.0, q0=q0))
    k_h, k_d = 2e4, 40.0
    for i in range(n_links):
        for s in (-1.0, 1.0):
            a_pt = (-L / 2, 0.0, s * w / 2)
            if i == 0:
                joints.append(dict(a=0, a_kind=0, a_vec=a_pt, b=-1, b_kind=0, b_vec=(0.0, 0.0, 0.0), k=k_h,
                                   t=(0.0, 0.0, z0 + s * w / 2)))
            else:
                joints.append(dict(a=i, a_kind=0, a_vec=a_pt, b=i - 1, b_kind=0, b_vec=(L / 2, 0.0, s * w / 2), k=k_h,
                                   t=(0.0, 0.0, 0.0)))
        # drive: the link's axis toward the parent's axis turned by theta_i (the world x axis for link 0)
        joints.append(dict(a=i, a_kind=1, a_vec=(1.0, 0.0, 0.0), b=(i - 1 if i else -1), b_kind=1,
                           b_vec=(1.0, 0.0, 0.0), k=k_d, t=(0.0, 0.0, 0.0) if i else (1.0, 0.0, 0.0)))
    nj = len(joints)
    joint_b = np.zeros((n_steps + 1, nj, 3))
    joint_t = np.zeros((n_steps + 1, nj, 3))
    for s in range(n_steps + 1):
        ramp = swing * min(1.0, s / max(1, n_steps // 2))
        for j, jt in enumerate(joints):
            joint_b[s, j] = jt["b_vec"]
            joint_t[s, j] = jt["t"]
        for i in range(n_links):
            th = ramp * (1.0 if i % 2 == 0 else -0.5)
            j = 3 * i + 2
            d = np.array([math.cos(th), math.sin(th), 0.0])
            if i == 0:
                joint_t[s, j] = d
            else:
                joint_b[s, j] = d
    gX = np.array([[-1.0, -1.0, 0.0], [2.0, -1.0, 0.0], [-1.0, 2.0, 0.0]])
    gT = np.array([[0, 1, 2]], np.int32)
    kin = [dict(X=gX, tris=gT)]
    kin_T = np.tile(translation((0.0, 0.0, 0.0)), (n_steps + 1, 1, 1, 1))
    if with_block:
        reach = L * n_links
        X, tets = grid_tets((reach - 8 * mm, 16 * mm, 0.4 * mm), 5 * mm, 2, 2, 2)
    else:
        X, tets = np.zeros((0, 3)), np.zeros((0, 4), np.int32)
    nt = len(tets)
    params = default_params(dt=1e-2, dhat=0.5 * mm, mu=0.2, n_steps=n_steps)
    params.update(param_overrides)
    return dict(
        name=f"jointed_arm_{n_links}links",
        fem_X=X, fem_tets=tets,
        fem_logE=np.full(nt, math.log(1e5)), fem_nu=np.full(nt, 0.4), fem_rho=np.full(nt, 1000.0),
        fem_body=np.zeros(nt, np.int32),
        kin=kin, kin_T=kin_T, abd=abd,
        stitch_v=np.zeros(0, np.int32), stitch_b=np.zeros(0, np.int32), stitch_X=np.zeros((0, 3)),
        joints=joints, joint_b=joint_b, joint_t=joint_t,
        gravity=np.array([0.0, 0.0, -9.81 if gravity else 0.0]),
        params=params,
    )


def abd_box_drop(n_steps: int = 6, mu: float = 0.3, **param_overrides) -> dict:
    """A 20 mm rigid (ABD) box, slightly tilted, falling onto a fixed ground triangle, beside a
    soft 2 x 2 x 2 mm block resting on the same ground (ABD-kinematic and FEM-kinematic contact)."""
    mm = 1e-3
    bX, bT = box_surface((-10 * mm, -10 * mm, -10 * mm), (10 * mm, 10 * mm, 10 * mm))
    R = rot_x(0.03) @ rot_y(0.02)
    q0 = np.concatenate([[0.0, 0.0, 10.9 * mm], R[:, 0], R[:, 1], R[:, 2]])
    X, tets = grid_tets((15 * mm, -1 * mm, 0.25 * mm), 1 * mm, 2, 2, 2)
    nt = len(tets)
    gX = np.array([[-50 * mm, -50 * mm, 0.0], [250 * mm, -50 * mm, 0.0], [-50 * mm, 250 * mm, 0.0]])
    kin_T = np.tile(translation((0, 0, 0)), (n_steps + 1, 1, 1, 1))
    sv, sb, sx = _empty_stitch()
    params = default_params(dt=1e-2, dhat=0.5 * mm, mu=mu, n_steps=n_steps)
    params.update(param_overrides)
    return dict(
        name="abd_box_drop",
        fem_X=X, fem_tets=tets,
        fem_logE=np.full(nt, math.log(1e5)), fem_nu=np.full(nt, 0.4), fem_rho=np.full(nt, 1000.0),
        fem_body=np.zeros(nt, np.int32),
        kin=[dict(X=gX, tris=np.array([[0, 1, 2]], np.int32))], kin_T=kin_T,
        abd=[dict(X=bX, tris=bT, rho=1000.0, q0=q0)],
        stitch_v=sv, stitch_b=sb, stitch_X=sx,
        gravity=np.array([0.0, 0.0, -9.81]),
        params=params,
    )


def stitched_block(n_steps: int = 6, **param_overrides) -> dict:
    """A 4 x 4 x 4 mm soft block (2 mm cells) whose top vertices are stitched
    (Eq. 2) to a kinematic base that moves sideways and up; the block swings."""
    mm = 1e-3
    X, tets = grid_tets((-2 * mm, -2 * mm, 0.0), 2 * mm, 2, 2, 2)
    nt = len(tets)
    top = np.where(np.abs(X[:, 2] - 4 * mm) < 1e-9)[0].astype(np.int32)
    bX, bT = box_surface((-3 * mm, -3 * mm, 4.6 * mm), (3 * mm, 3 * mm, 6 * mm))
    kin_T = np.zeros((n_steps + 1, 1, 3, 4))
    for s in range(n_steps + 1):
        kin_T[s, 0] = translation((0.2 * mm * s, 0.0, 0.1 * mm * s))
    params = default_params(dt=1e-2, dhat=0.3 * mm, mu=0.0, n_steps=n_steps)
    params.update(param_overrides)
    return dict(
        name="stitched_block",
        fem_X=X, fem_tets=tets,
        fem_logE=np.full(nt, math.log(1e5)), fem_nu=np.full(nt, 0.45), fem_rho=np.full(nt, 1100.0),
        fem_body=np.zeros(nt, np.int32),
        kin=[dict(X=bX, tris=bT)], kin_T=kin_T, abd=[],
        stitch_v=top, stitch_b=np.zeros(len(top), np.int32), stitch_X=X[top].copy(),
        gravity=np.array([0.0, 0.0, -9.81]),
        params=params,
    )


def ellipsoid_or_box_object(rng: SplitMix64, tris_lo=1000, tris_hi=8000, size_lo=20e-3, size_hi=60e-3):
    """Seeded rigid object: an ellipsoid or a box (probability 1/2 each), 1k-8k triangles, 20-60 mm."""
    u = rng.uniform(5)
    ntris = int(tris_lo + (tris_hi - tris_lo) * u[0])
    dims = size_lo + (size_hi - size_lo) * np.sort(u[1:4])[::-1]
    if u[4] < 0.5:
        n_lon = max(8, int(round(math.sqrt(ntris * 1.6 / 2))))
        n_lat = max(4, int(round(ntris / (2 * n_lon))) + 1)
        X, T = uv_ellipsoid(0.5 * dims[0], 0.5 * dims[1], 0.5 * dims[2], n_lat, n_lon)
        vol = math.pi / 6 * dims[0] * dims[1] * dims[2]
    else:
        n = max(2, int(round(math.sqrt(ntris / 12))))
        X, T = subdivided_box(-0.5 * dims, 0.5 * dims, n)
        vol = float(dims[0] * dims[1] * dims[2])
    return X, T, vol, dims


def translate_scene(sc: dict, offset) -> dict:
    """The same scene moved rigidly by `offset` (FEM rest/initial positions, ABD poses, kinematic transforms)."""
    off = np.asarray(offset, dtype=np.float64)
    sc = dict(sc)
    sc["fem_X"] = sc["fem_X"] + off
    sc["abd"] = [dict(a, q0=np.concatenate([a["q0"][:3] + off, a["q0"][3:]])) for a in sc.get("abd", [])]
    kin_T = sc["kin_T"].copy()
    kin_T[..., 3] += off
    sc["kin_T"] = kin_T
    return sc


def batched_grasps(n_scenes: int = 64, seed0: int = 0, n_steps: int = 200, tets_lo=5000, tets_hi=40000,
                   spacing: float = 1.2) -> list:
    """Independent grasp scenes for batched data generation.

    Scene k (seed seed0 + k): two fin-ray fingertips with a tet count drawn
    log-uniformly in [tets_lo, tets_hi] (the voxel size is chosen to match),
    a seeded rigid object (ellipsoid or box, 1k-8k triangles, 20-60 mm, ABD,
    0.1 kg), a random approach pose (yaw in [0, 2 pi), offset +/- 10 mm), and
    the close-and-lift trajectory of the single-scene grasp; no arm links.
    FP32-PCG / FP64-barrier configuration, dt = 5 ms, at most 500 Newton
    iterations per step.  Scene k is translated
    to grid cell (k mod 8, k div 8) with `spacing` metres between cells; a
    rigid translation leaves each scene's motion unchanged."""
    mm = 1e-3
    out = []
    base_tets = 47472 / 2  # one tip at 1.25 mm cells
    for k in range(n_scenes):
        rng = SplitMix64(seed0 + 1000 + k)
        u = rng.uniform(4)
        tets = math.exp(math.log(tets_lo) + (math.log(tets_hi) - math.log(tets_lo)) * u[0])
        cell = 1.25e-3 * (base_tets / tets) ** (1.0 / 3.0)
        sc = arm_gripper_grasp(seed0 + k, n_steps=n_steps, tip_cell=cell, link_tris=8, obj_tris=1000)
        # replace the object and drop the arm links
        oX, oT, vol, dims = ellipsoid_or_box_object(rng)
        half_h = 0.5 * float(oX[:, 2].max() - oX[:, 2].min())
        yaw = 2 * math.pi * u[1]
        R = rot_z(yaw)
        off = (2 * u[2:4] - 1) * 10 * mm
        q0 = np.concatenate([[off[0], off[1], half_h + 0.3 * mm], R[:, 0], R[:, 1], R[:, 2]])
        sc["abd"] = [dict(X=oX, tris=oT, rho=0.1 / vol, q0=q0)]
        # keep ground and finger bases (bodies 0..2); arm links are not part of the batched scenes
        sc["kin"] = sc["kin"][:3]
        sc["kin_T"] = sc["kin_T"][:, :3].copy()
        # open the fingers so that they clear the object: the object's half width along y
        half_w = 0.5 * float((oX @ R.T)[:, 1].max() - (oX @ R.T)[:, 1].min()) + abs(off[1])
        shift = max(0.0, half_w + 0.8 * mm - 25.8 * mm)
        X = sc["fem_X"].copy()
        X[:, 1] += np.sign(X[:, 1]) * shift
        sc["fem_X"] = X
        sc["stitch_X"] = sc["stitch_X"].copy()
        for s in range(sc["kin_T"].shape[0]):
            sc["kin_T"][s, 1, 1, 3] += shift
            sc["kin_T"][s, 2, 1, 3] -= shift
        sc["name"] = f"batched_grasp_{k}_{len(sc['fem_tets'])}tet"
        # some random poses meet lift steps where the projected Newton iteration converges slowly (full
        # steps, about 300 iterations; scene 14 at step 138): a larger cap than the single-scene default
        sc["params"] = dict(sc["params"], max_newton=500)
        # scenes sit on an 8-wide grid, `spacing` apart, so that their ground quads do not overlap
        out.append(translate_scene(sc, ((k % 8) * spacing, (k // 8) * spacing, 0.0)) if spacing else sc)
    return out


def voxel_cylinder(r, h, cell, z0=0.0):
    """Tet mesh of a vertical cylinder (radius r, height h, bottom at z0): the
    cells of a regular grid that lie wholly inside the circle, 6 tets each."""
    n = int(math.ceil(2 * r / cell))
    nz = int(round(h / cell))
    X, T = grid_tets((-0.5 * n * cell, -0.5 * n * cell, z0), cell, n, n, nz)
    ci = np.arange(n * n * nz)
    ii, jj = ci % n, (ci // n) % n
    xc = (ii + 0.5) * cell - 0.5 * n * cell
    yc = (jj + 0.5) * cell - 0.5 * n * cell
    ax, ay = np.abs(xc) + 0.5 * cell, np.abs(yc) + 0.5 * cell
    keep = ax * ax + ay * ay <= r * r
    T = T[np.repeat(keep, 6)]
    used = np.unique(T)
    remap = -np.ones(len(X), np.int64)
    remap[used] = np.arange(len(used))
    return morton_order(X[used], remap[T].astype(np.int32))


def soft_gripper_cylinder(seed: int = 0, n_steps: int = 300, tip_cell=1.25e-3, cyl_cell=2.15e-3,
                          close_per_step=0.05e-3, cyl_r=25e-3, cyl_h=60e-3, close_steps=200, base_tris=1000,
                          **param_overrides) -> dict:
    """The two fin-ray fingertips of the arm-gripper grasp squeeze a deformable
    Neo-Hookean cylinder (r = 25 mm, h = 60 mm, about 60k tets, E = 5e4 Pa,
    nu = 0.4, rho = 1100 assumed) resting on the ground quad; no arm links and
    no rigid object.  The fingertips start 0.8 mm from the cylinder; the
    finger bases close `close_per_step` (0.05 mm) per step for 200 steps
    (10 mm in all), then hold.  dt = 5 ms, dhat = 0.5 mm, mu = 0.6.  The
    cylinder's size and voxel size, the closing schedule and the base
    resolution are parameters (the reduced scene uses them)."""
    mm = 1e-3
    sc = arm_gripper_grasp(seed, n_steps=n_steps, tip_cell=tip_cell, link_tris=8, obj_tris=1000, base_tris=base_tris,
                           **param_overrides)
    cX, cT = voxel_cylinder(cyl_r, cyl_h, cyl_cell, z0=0.3 * mm)
    n_tip_v, n_tip_t = len(sc["fem_X"]), len(sc["fem_tets"])
    # move the fingertips (and their bases) in to 0.8 mm from the voxel surface
    shift = 25 * mm - float(np.abs(cX[:, 1]).max())
    tX = sc["fem_X"].copy()
    tX[:, 1] -= np.sign(tX[:, 1]) * shift
    X = np.concatenate([tX, cX])
    tets = np.concatenate([sc["fem_tets"], cT + n_tip_v])
    nt_c = len(cT)
    sc["fem_X"] = X
    sc["fem_tets"] = tets
    sc["fem_logE"] = np.concatenate([sc["fem_logE"], np.full(nt_c, math.log(5e4))])
    sc["fem_nu"] = np.concatenate([sc["fem_nu"], np.full(nt_c, 0.4)])
    sc["fem_rho"] = np.concatenate([sc["fem_rho"], np.full(nt_c, 1100.0)])
    sc["fem_body"] = np.concatenate([sc["fem_body"], np.full(nt_c, 2, np.int32)])
    sc["abd"] = []
    sc["kin"] = sc["kin"][:3]
    kin_T = sc["kin_T"][:, :3].copy()
    b, gap = 25 * mm - shift, 0.8 * mm
    z_top = kin_T[0, 1, 2, 3]
    for s in range(n_steps + 1):
        close = min(s, close_steps) * close_per_step
        kin_T[s, 1, :, 3] = (0.0, b + gap - close, z_top)
        kin_T[s, 2, :, 3] = (0.0, -(b + gap - close), z_top)
    sc["kin_T"] = kin_T
    sc["name"] = f"soft_gripper_cylinder_{len(tets)}tet"
    assert n_tip_t + nt_c == len(tets)
    return sc


def soft_gripper_cylinder_reduced(seed: int = 0, n_steps: int = 12, **param_overrides) -> dict:
    """The soft-gripper squeeze at a resolution the CPU oracle steps in seconds: 3 mm fingertip voxels, a
    deformable cylinder of radius 15 mm and height 30 mm in 3.75 mm voxels (E = 5e4 Pa, nu = 0.4) on the
    ground quad, finger bases of about 100 triangles closing 0.3 mm per step for 10 steps, then holding."""
    sc = soft_gripper_cylinder(seed, n_steps=n_steps, tip_cell=3.0e-3, cyl_cell=3.75e-3, close_per_step=0.3e-3,
                               cyl_r=15e-3, cyl_h=30e-3, close_steps=10, base_tris=100, **param_overrides)
    sc["name"] = f"soft_gripper_cylinder_reduced_{len(sc['fem_tets'])}tet"
    return sc
