"""Path tracer of the simulated frames with the shadow-receiving background material (§III-D.2, §III-D.3,
Eq. 7).  CPU: the oracle against closed forms (Eq. 7 at full and zero visibility, the linear penumbra of a
half-plane occluder, the direct light from a large area light on a diffuse floor).  GPU: the CUDA frame
equals the oracle's frame pixel by pixel."""
import math

import numpy as np
import pytest

from oracle import render as ro

CTEX = np.array([0.6, 0.4, 0.2], np.float32)


def quad(c, u, v):
    """Two triangles of the parallelogram c +- u +- v (normal along u x v)."""
    c, u, v = (np.asarray(a, np.float64) for a in (c, u, v))
    X = np.array([c - u - v, c + u - v, c + u + v, c - u + v])
    return X, np.array([[0, 1, 2], [0, 2, 3]])


class Builder:
    def __init__(self):
        self.X, self.T, self.types, self.rgb = [], [], [], []
        self.n = 0

    def add(self, Xq, Tq, mtype, rgb):
        self.X.append(Xq)
        self.T.append(Tq + self.n)
        self.n += len(Xq)
        self.types += [mtype] * len(Tq)
        self.rgb += [rgb] * len(Tq)

    def arrays(self):
        return (np.concatenate(self.X), np.concatenate(self.T).astype(np.int32), np.asarray(self.types, np.int32),
                np.asarray(self.rgb, np.float32))


H = 2.0
A = 0.25


def penumbra_scene(occluder=True, light_half=A):
    b = Builder()
    b.add(*quad((0, 0, 0), (5, 0, 0), (0, 5, 0)), ro.BACKGROUND, CTEX)
    # emitter facing down (normal -z); two-sided emitters make its orientation irrelevant
    b.add(*quad((0, 0, H), (light_half, 0, 0), (0, light_half, 0)), ro.EMISSIVE, [5.0, 5.0, 5.0])
    if occluder:
        b.add(*quad((-5.0, 0, H / 2), (5.0, 0, 0), (0, 5.0, 0)), ro.DIFFUSE, [0.5, 0.5, 0.5])
    return b.arrays()


def low_camera(w=24, h=16):
    # below the occluder's height, looking at the origin from +x
    return ro.camera((1.0, 0.0, H / 4), (0.0, 0.0, 0.0), (0, 0, 1), 20.0, w, h)


def hit_x(cam):
    """x of the background point seen through every pixel centre (ray / plane z = 0)."""
    c, w, h = cam
    eye, f, r, u, tf = c[:3], c[3:6], c[6:9], c[9:12], c[12]
    xs = np.zeros((h, w))
    for py in range(h):
        for px in range(w):
            sx = ((px + 0.5) / w * 2 - 1) * tf * (w / h)
            sy = (1 - (py + 0.5) / h * 2) * tf
            d = f + sx * r + sy * u
            t = -eye[2] / d[2]
            xs[py, px] = eye[0] + t * d[0]
    return xs


@pytest.mark.parametrize("lam", [0.0, 0.5, 1.0])
def test_background_unshadowed_keeps_its_texture(lam):
    """V = 1 everywhere (no occluder): Eq. 7 gives C_tex exactly, whatever lambda_s."""
    X, T, ty, rgb = penumbra_scene(occluder=False)
    img = ro.render(X, T, ty, rgb, low_camera(), spp=2, n_shadow=4, lambda_s=lam)
    assert np.array_equal(img, np.broadcast_to(CTEX, img.shape))


def test_lambda_zero_ignores_shadows():
    X, T, ty, rgb = penumbra_scene()
    img = ro.render(X, T, ty, rgb, low_camera(), spp=2, n_shadow=4, lambda_s=0.0)
    assert np.array_equal(img, np.broadcast_to(CTEX, img.shape))


def test_half_plane_penumbra_is_linear():
    """A half-plane occluder (x < 0) halfway up to a square light of half-width a: the segment from the
    background point (x, y, 0) to the light point (lx, ly, H) crosses the occluder's plane at x + (lx - x)/2,
    so the point sees the light where lx >= -x: V(x) = (a + x) / 2a (clamped), and Eq. 7 darkens the texture
    by lambda_s (1 - V)."""
    lam = 0.8
    X, T, ty, rgb = penumbra_scene()
    cam = low_camera(32, 16)
    img = ro.render(X, T, ty, rgb, cam, spp=16, n_shadow=32, lambda_s=lam)
    xs = hit_x(cam)
    V = np.clip((A + xs) / (2 * A), 0.0, 1.0)
    expect = (1 - lam * (1 - V))[..., None] * CTEX
    # fully lit / fully shadowed pixels are exact; the penumbra matches within the Monte Carlo error
    lit, dark = xs > A + 0.02, xs < -A - 0.02
    assert lit.any() and dark.any()
    assert np.allclose(img[lit], CTEX, atol=0) and np.allclose(img[dark], (1 - lam) * CTEX, atol=1e-7)
    pen = ~lit & ~dark
    err = np.abs(img[pen] - expect[pen]).mean() / CTEX.mean()
    assert err < 0.03, err


def corner_form_factor(a, b):
    """Form factor from a differential area to a parallel rectangle a x b (in units of the height) above
    one of its corners."""
    return (a / math.sqrt(1 + a * a) * math.atan(b / math.sqrt(1 + a * a)) +
            b / math.sqrt(1 + b * b) * math.atan(a / math.sqrt(1 + b * b))) / (2 * math.pi)


def test_diffuse_floor_under_square_light():
    """Direct light only (max_depth 0): a Lambertian floor of albedo rho under a square emitter of radiance
    Le and half-width s at height h reflects rho Le F, F the form factor of the square seen from the point
    (four corner rectangles of s x s)."""
    rho, Le, s, h = 0.7, 3.0, 0.5, 0.4
    b = Builder()
    b.add(*quad((0, 0, 0), (3, 0, 0), (0, 3, 0)), ro.DIFFUSE, [rho] * 3)
    b.add(*quad((0, 0, h), (s, 0, 0), (0, s, 0)), ro.EMISSIVE, [Le] * 3)
    X, T, ty, rgb = b.arrays()
    cam = ro.camera((0.0, 0.0, 0.2), (0.0, 0.0, 0.0), (0, 1, 0), 2.0, 4, 4)  # a tiny patch around the centre
    img = ro.render(X, T, ty, rgb, cam, spp=4096, max_depth=0, n_shadow=0)
    F = 4 * corner_form_factor(s / h, s / h)
    assert abs(img.mean() - rho * Le * F) <= 0.02 * rho * Le * F, (img.mean(), rho * Le * F)


def mixed_scene():
    """Every material: a textured background (per-triangle C_tex), diffuse boxes, a transparent sheet, two
    area lights."""
    b = Builder()
    r = np.random.default_rng(4)
    for i in range(4):
        for j in range(4):
            Xq, Tq = quad((-1.5 + i, -1.5 + j, 0.0), (0.5, 0, 0), (0, 0.5, 0))
            b.add(Xq, Tq, ro.BACKGROUND, r.uniform(0.2, 0.9, 3))
    for k in range(3):
        c = np.array([-0.6 + 0.6 * k, 0.1 * k, 0.3])
        for ax in range(3):
            for sgn in (-1, 1):
                n = np.zeros(3); n[ax] = sgn * 0.2
                u = np.zeros(3); u[(ax + 1) % 3] = 0.2
                v = np.zeros(3); v[(ax + 2) % 3] = 0.2
                Xq, Tq = quad(c + n, u if sgn > 0 else -u, v)
                b.add(Xq, Tq, ro.DIFFUSE, r.uniform(0.3, 0.9, 3))
    b.add(*quad((0.0, -0.3, 0.7), (0.8, 0, 0), (0, 0, 0.3)), ro.TRANSPARENT, [0.8, 0.9, 0.7])
    b.add(*quad((-0.8, 0.5, 2.0), (0.3, 0, 0), (0, 0.3, 0)), ro.EMISSIVE, [4.0, 4.0, 3.5])
    b.add(*quad((0.9, -0.6, 1.8), (0.2, 0, 0), (0, 0.2, 0)), ro.EMISSIVE, [3.0, 3.5, 4.0])
    return b.arrays()


@pytest.mark.gpu
def test_gpu_frame_equals_oracle_frame():
    torch = pytest.importorskip("torch")
    from paper_2609_25653_b300 import ipcsim
    X, T, ty, rgb = mixed_scene()
    cam = ro.camera((0.0, -3.5, 2.2), (0.0, 0.0, 0.3), (0, 0, 1), 45.0, 40, 30)
    P = dict(spp=4, max_depth=2, n_shadow=4, lambda_s=0.7, eps=1e-5, seed=11)
    ref = ro.render(X, T, ty, rgb, cam, **P)
    r = ipcsim.Renderer(T, ty, rgb, len(X))
    img = r.render(torch.as_tensor(X, device="cuda"), cam, **P)
    torch.cuda.synchronize()
    got = img.cpu().numpy()
    assert got.shape == ref.shape
    assert np.count_nonzero(got != ref) <= 2, np.argwhere(got != ref)[:10]
    assert np.max(np.abs(got - ref)) <= 1e-6 * max(1.0, float(np.abs(ref).max()))
    assert ref.max() > 0.1


@pytest.mark.gpu
def test_gpu_frame_of_simulated_grasp_equals_oracle():
    """A frame of the reduced arm-gripper grasp (every simulated surface, the background stand-in with
    Eq. 7, two area lights).  The simulator's vertex positions (ABD vertices p + A xbar with the device's
    fused multiply-adds) agree with the oracle's to rounding; both renderers then take the oracle's."""
    torch = pytest.importorskip("torch")
    from oracle import ipc as orc
    from paper_2609_25653_b300 import ipcsim, scenes
    sc = scenes.arm_gripper_grasp_reduced(0, n_steps=2)
    sim = ipcsim.Simulator(sc)
    S = orc.Scene(sc)
    _, tris_s, _ = sim.surface()
    extra, tris, types, rgb, cam = scenes.render_setup(sc, tris_s, sim.nv)
    X = np.concatenate([S.positions(S.z0), extra])
    xs = sim.positions().cpu().numpy()
    assert np.abs(xs - X[:sim.nv]).max() <= 1e-15 * np.abs(X).max()
    xv = torch.as_tensor(X, device="cuda").contiguous()
    c, _, _ = cam
    small = (c, 48, 27)
    P = dict(spp=2, max_depth=2, n_shadow=4, lambda_s=0.8, eps=1e-5, seed=3)
    ref = ro.render(X, tris, types, rgb, small, **P)
    got = ipcsim.Renderer(tris, types, rgb, len(X)).render(xv, small, **P).cpu().numpy()
    assert np.count_nonzero(got != ref) <= 3, np.argwhere(got != ref)[:10]
    assert np.max(np.abs(got - ref)) <= 1e-6 * float(np.abs(ref).max())
