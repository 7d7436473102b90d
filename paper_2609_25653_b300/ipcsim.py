"""Python binding of the ipcsim C ABI (include/ipcsim.h).

Argument marshalling only: every step of the IPC path runs in the CUDA
library.  There is no CPU fallback; loading fails loudly when the library
has not been built.  Device buffers are torch CUDA tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libipcsim.so")

dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int)
vp = C.c_void_p

IPC_OK = 0
STATUS = {0: "IPC_OK", -1: "IPC_ERR_ARG", -2: "IPC_ERR_INVERTED", -3: "IPC_ERR_INTERSECTING",
          -4: "IPC_ERR_NEWTON_MAXIT", -5: "IPC_ERR_PCG", -6: "IPC_ERR_LS_STALL", -7: "IPC_ERR_NAN",
          -8: "IPC_ERR_BVH_OVERFLOW", -9: "IPC_ERR_CUDA", -10: "IPC_ERR_CAPACITY"}
PREC_FP64, PREC_MIXED = 0, 1
BROAD_LBVH, BROAD_ALL_PAIRS = 0, 1
PRECOND_TWO_LEVEL, PRECOND_BLOCK_JACOBI = 0, 1


class SceneDesc(C.Structure):
    _fields_ = [
        ("n_fem_verts", C.c_int), ("fem_X_host", dp), ("fem_V0_host", dp),
        ("n_tets", C.c_int), ("tets_host", ip), ("logE_host", dp), ("nu_host", dp), ("rho_host", dp),
        ("fem_body_host", ip),
        ("n_abd", C.c_int), ("abd_nverts_host", ip), ("abd_X_host", dp), ("abd_ntris_host", ip),
        ("abd_tris_host", ip), ("abd_rho_host", dp), ("abd_q0_host", dp),
        ("n_kin", C.c_int), ("kin_nverts_host", ip), ("kin_X_host", dp), ("kin_ntris_host", ip),
        ("kin_tris_host", ip), ("kin_T0_host", dp),
        ("n_stitch", C.c_int), ("stitch_v_host", ip), ("stitch_b_host", ip), ("stitch_X_host", dp),
        ("gravity", C.c_double * 3),
        ("n_joints", C.c_int), ("joint_body_host", ip), ("joint_kind_host", ip), ("joint_vec_host", dp),
        ("joint_k_host", dp), ("joint_t_host", dp),
    ]


class Params(C.Structure):
    _fields_ = [("dt", C.c_double), ("dhat", C.c_double), ("kappa", C.c_double), ("mu", C.c_double),
                ("eps_v", C.c_double), ("k_c", C.c_double), ("kappa_A", C.c_double), ("newton_tol", C.c_double),
                ("pcg_rtol", C.c_double), ("s_ccd", C.c_double), ("max_newton", C.c_int), ("max_pcg", C.c_int),
                ("precision", C.c_int), ("pair_capacity", C.c_int), ("broad_phase", C.c_int),
                ("pair_capacity_max", C.c_int), ("preconditioner", C.c_int), ("coarse_rebuild", C.c_int),
                ("kappa_adaptive", C.c_int), ("kappa_dmin", C.c_double), ("kappa_max_factor", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class TorchAllocator:
    """The simulator's device memory from PyTorch's caching allocator (sim_create_with_allocator).

    Keeps the ctypes callbacks alive for the simulator's lifetime and counts the calls."""

    def __init__(self):
        import torch
        self.allocs = 0
        self.frees = 0
        self.live = {}

        def _alloc(nbytes, stream, ctx):
            try:
                dev = torch.cuda.current_device()
                p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, int(stream or 0))
            except Exception:
                return None
            self.allocs += 1
            self.live[p] = nbytes
            return p

        def _free(ptr, stream, ctx):
            if ptr:
                self.frees += 1
                self.live.pop(ptr, None)
                torch.cuda.caching_allocator_delete(ptr)

        self._alloc = ALLOC_FN(_alloc)
        self._free = FREE_FN(_free)
        self.struct = Allocator(self._alloc, self._free, None)


class RenderScene(C.Structure):
    _fields_ = [("n_verts", C.c_int), ("n_tris", C.c_int), ("tris_host", ip), ("type_host", ip),
                ("rgb_host", C.POINTER(C.c_float))]


class Camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("fwd", C.c_float * 3), ("right", C.c_float * 3), ("up", C.c_float * 3),
                ("tan_half_fov", C.c_float), ("width", C.c_int), ("height", C.c_int)]


class RenderParams(C.Structure):
    _fields_ = [("spp", C.c_int), ("max_depth", C.c_int), ("n_shadow", C.c_int), ("lambda_s", C.c_float),
                ("eps", C.c_float), ("seed", C.c_ulonglong)]


class StepStats(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int), ("pcg_iters_total", C.c_int),
                ("pcg_iters_max", C.c_int), ("n_pairs_max", C.c_int), ("n_friction_pairs", C.c_int),
                ("n_ccd_max", C.c_int), ("ls_halvings", C.c_int), ("alpha_min", C.c_double),
                ("min_dist", C.c_double), ("energy_end", C.c_double), ("pnorm_end", C.c_double),
                ("pcg_unconverged", C.c_int), ("pcg_fallbacks", C.c_int), ("kappa_end", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# every exported symbol of the C ABI and its (argtypes, restype)
SIGNATURES = {
    "sim_create": ([C.POINTER(SceneDesc), C.POINTER(Params), vp, C.POINTER(vp)], C.c_int),
    "sim_create_batch": ([C.POINTER(SceneDesc), C.c_int, C.POINTER(Params), vp, C.POINTER(vp)], C.c_int),
    "sim_step": ([vp, dp, C.POINTER(StepStats)], C.c_int),
    "sim_get_state": ([vp, vp, vp, vp, vp, C.c_int], C.c_int),
    "sim_set_state": ([vp, vp, vp, vp, vp, C.c_int], C.c_int),
    "sim_sizes": ([vp, ip], C.c_int),
    "sim_scalars": ([vp, dp], C.c_int),
    "sim_last_error": ([vp], C.c_char_p),
    "sim_destroy": ([vp], None),
    "sim_eval_elastic": ([vp, vp, C.c_int, vp, vp, vp], C.c_int),
    "sim_active_pairs": ([vp, vp, C.c_int, vp, vp, ip], C.c_int),
    "sim_surface": ([vp, ip, ip, ip], C.c_int),
    "sim_eval_barrier": ([vp, vp, C.c_int, vp, C.c_int, vp, vp, vp], C.c_int),
    "sim_ccd_alpha": ([vp, vp, vp, dp, ip], C.c_int),
    "sim_kernel_launches": ([], C.c_ulonglong),
    "sim_profile": ([vp, C.c_int], C.c_int),
    "sim_set_params": ([vp, dp, C.c_double], C.c_int),
    "sim_set_kinematic": ([vp, dp], C.c_int),
    "sim_tuning": ([vp, C.c_int, C.c_int, C.c_int, ip, C.POINTER(C.c_float)], C.c_int),
    "sim_eval_barrier_noalloc": ([vp, vp, C.c_int, vp, C.c_int, vp, vp, vp], C.c_int),
    "sim_step_many": ([C.POINTER(vp), C.c_int, C.POINTER(dp), C.POINTER(StepStats), ip], C.c_int),
    "sim_adjoint": ([vp, vp, vp, vp, dp, dp, vp, vp, vp, vp, vp, dp], C.c_int),
    "sim_set_joint_targets": ([vp, dp, dp], C.c_int),
    "sim_profile_read": ([vp, dp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)], C.c_int),
    "sim_pcg_partition": ([ip, C.c_int, C.c_int, C.c_int, ip, C.c_int, ip, ip, ip, ip, ip], C.c_int),
    "sim_pcg_residency": ([vp, C.c_int], C.c_int),
    "sim_coarse_info": ([vp, C.POINTER(C.c_longlong)], C.c_int),
    "sim_device_peaks": ([dp], C.c_int),
    "sim_create_with_allocator": ([C.POINTER(SceneDesc), C.c_int, C.POINTER(Params), C.POINTER(Allocator), vp,
                                   C.POINTER(vp)], C.c_int),
    "sim_memory": ([vp, C.POINTER(C.c_longlong)], C.c_int),
    "sim_dual_mesh_create": ([ip, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(vp)], C.c_int),
    "sim_dual_mesh_sizes": ([vp, C.POINTER(C.c_longlong)], C.c_int),
    "sim_dual_mesh_topology": ([vp, ip, ip, ip, dp], C.c_int),
    "sim_dual_mesh_apply": ([vp, vp, vp, vp], C.c_int),
    "sim_dual_mesh_last_error": ([], C.c_char_p),
    "sim_dual_mesh_destroy": ([vp], None),
    "sim_render_create": ([C.POINTER(RenderScene), C.POINTER(vp)], C.c_int),
    "sim_positions": ([vp, vp], C.c_int),
    "sim_render_frame": ([vp, vp, C.POINTER(Camera), C.POINTER(RenderParams), vp, vp], C.c_int),
    "sim_render_last_error": ([], C.c_char_p),
    "sim_render_destroy": ([vp], None),
}

PROFILE_STAGES = ["pcg", "elastic", "barrier", "cull", "ccd", "friction", "other", "pcg_setup"]


def load():
    """Load the built CUDA library (raises if it is missing: no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"ipcsim CUDA library not built: {LIB_PATH} (run paper_2609_25653_b300/build.py)")
        L = C.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def device_peaks() -> dict:
    """Measured FP64 and FP32 FMA rates of the current device, TFLOP/s (sim_device_peaks)."""
    out = (C.c_double * 2)()
    code = load().sim_device_peaks(out)
    if code != IPC_OK:
        raise IpcError(code, "sim_device_peaks failed")
    return {"fp64_tflops": out[0], "fp32_tflops": out[1]}


def kernel_launches() -> int:
    """Kernels launched by the CUDA library so far in this process."""
    return int(load().sim_kernel_launches())


def pcg_partition(row, nf: int, nab: int, grid: int, node_scene=None, n_scenes: int = 1, row_extra=None) -> dict:
    """The PCG's partition of the rows among `grid` CTAs (sim_pcg_partition; host only, no GPU)."""
    row = np.ascontiguousarray(row, dtype=np.int32)
    ns = None if node_scene is None else np.ascontiguousarray(node_scene, dtype=np.int32)
    ex = None if row_extra is None else np.ascontiguousarray(row_extra, dtype=np.int32)
    out4 = np.zeros(4, np.int32)
    seg = np.zeros(grid + 1, np.int32)
    abd_seg = np.zeros(grid + 1, np.int32)
    cta_scene = np.zeros(grid, np.int32)
    as_ip = lambda a: a.ctypes.data_as(ip)
    st = load().sim_pcg_partition(as_ip(row), nf, nab, grid, None if ns is None else as_ip(ns), n_scenes,
                                  None if ex is None else as_ip(ex), as_ip(out4), as_ip(seg), as_ip(abd_seg),
                                  as_ip(cta_scene))
    if st != 0:
        raise ValueError(f"sim_pcg_partition failed ({st})")
    n_fem, n_abd = int(out4[0]), int(out4[1])
    return dict(n_fem_ctas=n_fem, n_abd_ctas=n_abd, n_solves=int(out4[2]), max_rows=int(out4[3]),
                seg=seg[:n_fem + 1].copy(), abd_seg=abd_seg[:n_abd + 1].copy(), cta_scene=cta_scene)


class IpcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(t):
    """Device pointer of a torch CUDA tensor (or None)."""
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def make_params(p: dict, precision=PREC_FP64) -> Params:
    return Params(dt=p["dt"], dhat=p["dhat"], kappa=p.get("kappa", 0.0), mu=p["mu"], eps_v=p["eps_v"],
                  k_c=p.get("k_c", 0.0), kappa_A=p.get("kappa_A", 1e8), newton_tol=p["newton_tol"],
                  pcg_rtol=p.get("pcg_rtol", 1e-4), s_ccd=p.get("s_ccd", 0.1), max_newton=int(p.get("max_newton", 100)),
                  max_pcg=int(p.get("max_pcg", 0)), precision=int(precision), pair_capacity=int(p.get("pair_capacity", 0)),
                  broad_phase=int(p.get("broad_phase", BROAD_LBVH)), pair_capacity_max=int(p.get("pair_capacity_max", 0)),
                  preconditioner=int(p.get("preconditioner", PRECOND_TWO_LEVEL)),
                  coarse_rebuild=int(p.get("coarse_rebuild", 0)), kappa_adaptive=int(p.get("kappa_adaptive", 0)),
                  kappa_dmin=float(p.get("kappa_dmin", 1e-2)), kappa_max_factor=float(p.get("kappa_max_factor", 100.0)))


def _fill_desc(d, scene, keep):
    """Fill one SceneDesc from a scene dictionary (the arrays are kept alive in `keep`)."""
    def arr_d(a):
        a = _f64(a)
        keep.append(a)
        return a.ctypes.data_as(dp)

    def arr_i(a):
        a = _i32(a)
        keep.append(a)
        return a.ctypes.data_as(ip)

    X = _f64(scene["fem_X"])
    d.n_fem_verts = X.shape[0]
    d.fem_X_host = arr_d(X)
    d.fem_V0_host = arr_d(scene["fem_V0"]) if "fem_V0" in scene else None
    d.n_tets = len(scene["fem_tets"])
    d.tets_host = arr_i(scene["fem_tets"])
    d.logE_host = arr_d(scene["fem_logE"])
    d.nu_host = arr_d(scene["fem_nu"])
    d.rho_host = arr_d(scene["fem_rho"])
    d.fem_body_host = arr_i(scene["fem_body"]) if "fem_body" in scene else None
    abd = scene.get("abd", [])
    d.n_abd = len(abd)
    if abd:
        d.abd_nverts_host = arr_i([a["X"].shape[0] for a in abd])
        d.abd_X_host = arr_d(np.concatenate([a["X"] for a in abd]))
        d.abd_ntris_host = arr_i([len(a["tris"]) for a in abd])
        d.abd_tris_host = arr_i(np.concatenate([a["tris"] for a in abd]))
        d.abd_rho_host = arr_d([a["rho"] for a in abd])
        d.abd_q0_host = arr_d(np.stack([a["q0"] for a in abd]))
    kin = scene.get("kin", [])
    d.n_kin = len(kin)
    if kin:
        d.kin_nverts_host = arr_i([k["X"].shape[0] for k in kin])
        d.kin_X_host = arr_d(np.concatenate([k["X"] for k in kin]))
        d.kin_ntris_host = arr_i([len(k["tris"]) for k in kin])
        d.kin_tris_host = arr_i(np.concatenate([k["tris"] for k in kin]))
        d.kin_T0_host = arr_d(scene["kin_T"][0].reshape(-1, 12))
    sv = scene.get("stitch_v", np.zeros(0, np.int32))
    d.n_stitch = len(sv)
    if len(sv):
        d.stitch_v_host = arr_i(sv)
        d.stitch_b_host = arr_i(scene["stitch_b"])
        d.stitch_X_host = arr_d(scene["stitch_X"])
    for k in range(3):
        d.gravity[k] = float(scene["gravity"][k])
    joints = scene.get("joints", [])
    d.n_joints = len(joints)
    if joints:
        d.joint_body_host = arr_i([[j["a"], j["b"]] for j in joints])
        d.joint_kind_host = arr_i([[j["a_kind"], j["b_kind"]] for j in joints])
        d.joint_vec_host = arr_d([[j["a_vec"], j["b_vec"]] for j in joints])
        d.joint_k_host = arr_d([j["k"] for j in joints])
        d.joint_t_host = arr_d([j.get("t", (0.0, 0.0, 0.0)) for j in joints])


def batch_scene(scenes):
    """Bookkeeping view of a batch (concatenated kinematic trajectories, first scene's parameters)."""
    n_steps = min(sc["kin_T"].shape[0] for sc in scenes)
    kin_T = np.concatenate([sc["kin_T"][:n_steps] for sc in scenes], axis=1)
    return dict(name=f"batch_{len(scenes)}", params=dict(scenes[0]["params"]), kin_T=kin_T,
                kin=[k for sc in scenes for k in sc.get("kin", [])], abd=[a for sc in scenes for a in sc.get("abd", [])],
                fem_X=np.concatenate([sc["fem_X"] for sc in scenes]),
                fem_tets=np.zeros((sum(len(sc["fem_tets"]) for sc in scenes), 4), np.int32),
                gravity=scenes[0]["gravity"])


class Simulator:
    """One scene on the GPU.  `scene` is a dictionary from paper_2609_25653_b300.scenes."""

    def __init__(self, scene: dict, precision=PREC_FP64, stream=None, _batch=None, allocator=None, **param_overrides):
        L = load()
        self.scene = scene
        p = dict(scene["params"])
        p.update(param_overrides)
        self.params = p
        keep = []
        scenes = _batch if _batch is not None else [scene]
        descs = (SceneDesc * len(scenes))()
        for i, sc in enumerate(scenes):
            _fill_desc(descs[i], sc, keep)
        par = make_params(p, precision)
        h = C.c_void_p()
        st = C.c_void_p(stream.cuda_stream if stream is not None else 0)
        self.allocator = allocator  # kept alive with the simulator
        if allocator is not None:
            code = L.sim_create_with_allocator(descs, len(scenes), C.byref(par), C.byref(allocator.struct), st,
                                               C.byref(h))
        elif _batch is None:
            code = L.sim_create(C.byref(descs[0]), C.byref(par), st, C.byref(h))
        else:
            code = L.sim_create_batch(descs, len(scenes), C.byref(par), st, C.byref(h))
        if code != IPC_OK:
            raise IpcError(code, L.sim_last_error(None).decode())
        self.h = h
        self.step_index = 0
        sz = (C.c_int * 9)()
        L.sim_sizes(h, sz)
        (self.nf, self.nt, self.nab, self.nkb, self.ntri, self.nedge, self.nsv, self.n_nodes, self.nnzb) = list(sz)
        self.nv = self.nf + sum(a["X"].shape[0] for sc in scenes for a in sc.get("abd", [])) + \
            sum(k["X"].shape[0] for sc in scenes for k in sc.get("kin", []))
        self.n_scenes = len(scenes)
        self._scenes = scenes
        self.nj = sum(len(s.get("joints", [])) for s in scenes)
        sc = (C.c_double * 4)()
        L.sim_scalars(h, sc)
        self.kappa, self.k_c, self.L, self.dhat = list(sc)

    @classmethod
    def batch(cls, scenes, precision=PREC_FP64, stream=None, **param_overrides):
        """One simulator advancing independent scenes together (sim_create_batch)."""
        return cls(batch_scene(scenes), precision=precision, stream=stream, _batch=list(scenes), **param_overrides)

    def close(self):
        if getattr(self, "h", None):
            load().sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, code):
        if code != IPC_OK:
            raise IpcError(code, load().sim_last_error(self.h).decode())

    def joint_targets(self, step):
        """The joints' b-side vectors and targets of trajectory step `step` (scene keys joint_b / joint_t,
        (n_steps + 1, n_joints, 3) each), all scenes concatenated; (None, None) without per-step targets."""
        if not self.nj or not any("joint_b" in s or "joint_t" in s for s in self._scenes):
            return None, None
        vb, t = [], []
        for s in self._scenes:
            jn = s.get("joints", [])
            if not jn:
                continue
            vb.append(_f64(s["joint_b"][step]) if "joint_b" in s else _f64([j["b_vec"] for j in jn]))
            t.append(_f64(s["joint_t"][step]) if "joint_t" in s else _f64([j.get("t", (0, 0, 0)) for j in jn]))
        return np.concatenate(vb).reshape(-1, 3), np.concatenate(t).reshape(-1, 3)

    def set_joint_targets(self, vec_b=None, t=None):
        """Drive targets of the joints for the following steps (sim_set_joint_targets): b-side body-frame
        vectors (n_joints, 3) and target offsets (n_joints, 3); None keeps."""
        a = None if vec_b is None else _f64(vec_b).reshape(-1)
        b = None if t is None else _f64(t).reshape(-1)
        for x in (a, b):
            if x is not None and x.size != 3 * self.nj:
                raise ValueError(f"joint targets need {3 * self.nj} values, got {x.size}")
        self._check(load().sim_set_joint_targets(self.h, None if a is None else a.ctypes.data_as(dp),
                                                 None if b is None else b.ctypes.data_as(dp)))

    def _trajectory_joint_targets(self, step):
        vb, t = self.joint_targets(step)
        if vb is not None:
            self.set_joint_targets(vb, t)

    def step(self, kin_T_next=None, raise_on_error=True, joint_targets=None):
        """Advance one step; kin_T_next (n_kin, 3, 4), joint_targets (vec_b, t).  Both default to the
        scene's trajectory."""
        if joint_targets is not None:
            self.set_joint_targets(*joint_targets)
        else:
            self._trajectory_joint_targets(self.step_index + 1)
        if kin_T_next is None and self.nkb:
            kin_T_next = self.scene["kin_T"][self.step_index + 1]
        T = _f64(kin_T_next).reshape(-1) if self.nkb else None
        stats = StepStats()
        code = load().sim_step(self.h, T.ctypes.data_as(dp) if T is not None else None, C.byref(stats))
        if code == IPC_OK:
            self.step_index += 1
        elif raise_on_error:
            self._check(code)
        return stats.as_dict()

    def get_state(self):
        x = np.zeros((self.nf, 3))
        v = np.zeros((self.nf, 3))
        q = np.zeros((self.nab, 12))
        qd = np.zeros((self.nab, 12))
        self._check(load().sim_get_state(self.h, x.ctypes.data_as(vp), v.ctypes.data_as(vp),
                                         q.ctypes.data_as(vp) if self.nab else None,
                                         qd.ctypes.data_as(vp) if self.nab else None, 0))
        return x, v, q, qd

    def positions(self, out=None):
        """All vertex positions (FEM | ABD surface | kinematic) of the current state, device (nv, 3)."""
        import torch
        if out is None:
            out = torch.empty((self.nv, 3), dtype=torch.float64, device="cuda")
        self._check(load().sim_positions(self.h, _ptr(out)))
        return out

    def get_state_device(self, x, v=None, q=None, qd=None):
        self._check(load().sim_get_state(self.h, _ptr(x), _ptr(v), _ptr(q), _ptr(qd), 1))

    def set_state(self, x=None, v=None, q=None, qd=None):
        arrs = [None if a is None else _f64(a) for a in (x, v, q, qd)]
        ptrs = [None if a is None else a.ctypes.data_as(vp) for a in arrs]
        self._check(load().sim_set_state(self.h, *ptrs, 0))

    # ---- parameters, DOF vectors and the adjoint ------------------------------
    @property
    def ndof(self):
        return 3 * self.n_nodes

    def set_params(self, logE=None, mu=None):
        """Per-tet ln E (host array) and friction coefficient for the following steps."""
        arr = None if logE is None else _f64(logE)
        self._check(load().sim_set_params(self.h, None if arr is None else arr.ctypes.data_as(dp),
                                          -1.0 if mu is None else float(mu)))
        if mu is not None:
            self.params["mu"] = float(mu)

    def set_kinematic(self, T):
        """Place the kinematic bodies at transforms T (n_kin, 3, 4)."""
        if self.nkb:
            arr = _f64(T).reshape(-1)
            self._check(load().sim_set_kinematic(self.h, arr.ctypes.data_as(dp)))

    def get_dofs(self):
        """(z, zd) as device tensors (n_nodes * 3): FEM vertices, then ABD q."""
        import torch
        z = torch.empty(self.ndof, dtype=torch.float64, device="cuda")
        zd = torch.empty(self.ndof, dtype=torch.float64, device="cuda")
        off = 8 * 3 * self.nf
        q = C.c_void_p(z.data_ptr() + off) if self.nab else None
        qd = C.c_void_p(zd.data_ptr() + off) if self.nab else None
        self._check(load().sim_get_state(self.h, _ptr(z), _ptr(zd), q, qd, 1))
        return z, zd

    def set_dofs(self, z, zd):
        z = z.contiguous()
        zd = zd.contiguous()
        off = 8 * 3 * self.nf
        q = C.c_void_p(z.data_ptr() + off) if self.nab else None
        qd = C.c_void_p(zd.data_ptr() + off) if self.nab else None
        self._check(load().sim_set_state(self.h, _ptr(z), _ptr(zd), q, qd, 1))

    def adjoint(self, z_t, zd_t, z_next, T_t, T_next, gz_next, gzd_next, glogE=None, step_next=None):
        """Backward of one step: returns (dL/dz_t, dL/dzd_t, glogE (accumulated), dL/dmu).  step_next: the
        trajectory index of z_next, whose joint targets are set first (scenes with per-step targets)."""
        import torch
        if step_next is not None:
            self._trajectory_joint_targets(step_next)
        gz_t = torch.empty(self.ndof, dtype=torch.float64, device="cuda")
        gzd_t = torch.empty(self.ndof, dtype=torch.float64, device="cuda")
        if glogE is None:
            glogE = torch.zeros(self.nt, dtype=torch.float64, device="cuda")
        gmu = C.c_double(0.0)
        Tt = _f64(T_t).reshape(-1) if self.nkb else None
        Tn = _f64(T_next).reshape(-1) if self.nkb else None
        self._check(load().sim_adjoint(self.h, _ptr(z_t.contiguous()), _ptr(zd_t.contiguous()), _ptr(z_next.contiguous()),
                                       Tt.ctypes.data_as(dp) if Tt is not None else None,
                                       Tn.ctypes.data_as(dp) if Tn is not None else None,
                                       _ptr(gz_next.contiguous()), _ptr(gzd_next.contiguous()), _ptr(gz_t), _ptr(gzd_t),
                                       _ptr(glogE), C.byref(gmu)))
        return gz_t, gzd_t, glogE, gmu.value

    def tuning(self, rowg=0, blocks_per_sm=0, autotune_next_step=False):
        """Set / read the PCG launch shape; returns ((rowg, blocks_per_sm), last autotuning times in ms)."""
        out = (C.c_int * 4)()
        ms = (C.c_float * 8)()
        self._check(load().sim_tuning(self.h, int(rowg), int(blocks_per_sm), int(bool(autotune_next_step)), out, ms))
        return (out[0], out[1]), list(ms)

    def memory(self):
        """(blocks from the caller's allocator, blocks from cudaMalloc, bytes held)."""
        out = (C.c_longlong * 3)()
        self._check(load().sim_memory(self.h, out))
        return tuple(out)

    def coarse_info(self):
        """(aggregates, solves, coarse unknowns of the largest solve, last build ok) of the two-level
        preconditioner."""
        out = (C.c_longlong * 4)()
        self._check(load().sim_coarse_info(self.h, out))
        return tuple(int(v) for v in out)

    def coarse_size(self):
        """Coarse unknowns of the largest solve of the last build (0 when the last build failed)."""
        a, s, n, ok = self.coarse_info()
        return n if ok else 0

    def pcg_residency(self, streamed: bool):
        """streamed=True: the PCG reads its operator from global memory in every iteration (never staged in
        shared memory); False: staged when every CTA's rows fit (default)."""
        self._check(load().sim_pcg_residency(self.h, int(bool(streamed))))

    def pcg_layout(self):
        """(CTAs, operator resident in shared memory) of the last PCG launch."""
        out = (C.c_int * 4)()
        self._check(load().sim_tuning(self.h, 0, 0, 0, out, None))
        return out[2], bool(out[3])

    def profile(self, enable=True, reset=True):
        """Per-stage CUDA-event accounting: on (cleared unless reset=False, which resumes it) or off."""
        self._check(load().sim_profile(self.h, (1 if reset else 2) if enable else 0))

    def profile_read(self):
        ms = (C.c_double * 8)()
        n = (C.c_longlong * 8)()
        w = (C.c_longlong * 4)()
        self._check(load().sim_profile_read(self.h, ms, n, w))
        stages = {PROFILE_STAGES[k]: dict(ms=ms[k], n=n[k]) for k in range(8)}
        work = dict(pcg_iters=w[0], pcg_pair_iters=w[1], pcg_fric_iters=w[2], bsr_blocks=w[3])
        return stages, work

    # ---- stage entry points (device tensors) ---------------------------------
    def surface(self):
        sv = np.zeros(self.nsv, np.int32)
        tris = np.zeros((self.ntri, 3), np.int32)
        edges = np.zeros((self.nedge, 2), np.int32)
        self._check(load().sim_surface(self.h, sv.ctypes.data_as(ip), tris.ctypes.data_as(ip), edges.ctypes.data_as(ip)))
        return sv, tris, edges

    def eval_elastic(self, x_dev, project=True, want_hess=True):
        import torch
        E = torch.zeros(1, dtype=torch.float64, device=x_dev.device)
        g = torch.zeros((self.nf, 3), dtype=torch.float64, device=x_dev.device)
        H = torch.zeros((self.nt, 12, 12), dtype=torch.float64, device=x_dev.device) if want_hess else None
        self._check(load().sim_eval_elastic(self.h, _ptr(x_dev), int(project), _ptr(E), _ptr(g), _ptr(H)))
        return E, g, H

    def active_pairs(self, xv_dev, cap=None):
        import torch
        cap = cap or max(1024, 4 * (self.nsv + self.nedge))
        while True:
            rec = torch.zeros((cap, 8), dtype=torch.int32, device=xv_dev.device)
            s = torch.zeros(cap, dtype=torch.float64, device=xv_dev.device)
            n = C.c_int()
            code = load().sim_active_pairs(self.h, _ptr(xv_dev), cap, _ptr(rec), _ptr(s), C.byref(n))
            if code == -10:
                cap = n.value
                continue
            self._check(code)
            return rec[:n.value], s[:n.value]

    def eval_barrier(self, xv_dev, rec_dev, project=True):
        import torch
        n = rec_dev.shape[0]
        E = torch.zeros(1, dtype=torch.float64, device=xv_dev.device)
        g = torch.zeros((self.n_nodes, 3), dtype=torch.float64, device=xv_dev.device)
        H = torch.zeros((max(n, 1), 12, 12), dtype=torch.float64, device=xv_dev.device)
        rec_dev = rec_dev.contiguous()
        self._check(load().sim_eval_barrier(self.h, _ptr(xv_dev), n, _ptr(rec_dev), int(project), _ptr(E), _ptr(g),
                                            _ptr(H)))
        return E, g, H[:n]

    def eval_barrier_noalloc(self, xv_dev, rec_dev, E, g, H, project=True):
        """sim_eval_barrier_noalloc: outputs go into the caller's tensors E (1), g (n_nodes, 3), H (n, 12, 12)."""
        rec_dev = rec_dev.contiguous()
        self._check(load().sim_eval_barrier_noalloc(self.h, _ptr(xv_dev), rec_dev.shape[0], _ptr(rec_dev), int(project),
                                                    _ptr(E), _ptr(g), _ptr(H)))

    def ccd_alpha(self, xv_dev, pv_dev):
        a = C.c_double()
        nc = C.c_int()
        self._check(load().sim_ccd_alpha(self.h, _ptr(xv_dev), _ptr(pv_dev), C.byref(a), C.byref(nc)))
        return a.value, nc.value


class DualMesh:
    """Render mesh of a deformable surface by L levels of Loop subdivision (Eqs. 5-6): W built once,
    X_f = W X_c per frame on the device.  upload=False keeps W on the host (inspection without a GPU)."""

    def __init__(self, tris, n_verts, levels, upload=True):
        L = load()
        t = _i32(tris)
        h = C.c_void_p()
        code = L.sim_dual_mesh_create(t.ctypes.data_as(ip), len(t), int(n_verts), int(levels), int(bool(upload)),
                                      C.byref(h))
        if code != IPC_OK:
            raise IpcError(code, L.sim_dual_mesh_last_error().decode())
        self.h = h
        sz = (C.c_longlong * 4)()
        L.sim_dual_mesh_sizes(h, sz)
        self.n_coarse, self.n_fine, self.n_fine_tris, self.nnz = (int(v) for v in sz)

    def topology(self):
        """(fine triangles, W as scipy CSR)."""
        import scipy.sparse as sp
        tris = np.zeros((self.n_fine_tris, 3), np.int32)
        row = np.zeros(self.n_fine + 1, np.int32)
        col = np.zeros(max(self.nnz, 1), np.int32)
        val = np.zeros(max(self.nnz, 1))
        load().sim_dual_mesh_topology(self.h, tris.ctypes.data_as(ip), row.ctypes.data_as(ip), col.ctypes.data_as(ip),
                                      val.ctypes.data_as(dp))
        return tris, sp.csr_matrix((val[:self.nnz], col[:self.nnz], row), shape=(self.n_fine, self.n_coarse))

    def apply(self, xc_dev, xf_dev=None, stream=None):
        """X_f = W X_c for device tensors; returns xf_dev ((N_fine, 3), allocated when None)."""
        import torch
        if xf_dev is None:
            xf_dev = torch.empty((self.n_fine, 3), dtype=torch.float64, device=xc_dev.device)
        st = C.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
        code = load().sim_dual_mesh_apply(self.h, _ptr(xc_dev.contiguous()), _ptr(xf_dev), st)
        if code != IPC_OK:
            raise IpcError(code, "sim_dual_mesh_apply failed")
        return xf_dev

    def close(self):
        if getattr(self, "h", None):
            load().sim_dual_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MAT_DIFFUSE, MAT_EMISSIVE, MAT_BACKGROUND, MAT_TRANSPARENT = 0, 1, 2, 3


class Renderer:
    """Headless path tracer of simulated frames (sim_render_*): triangles (n, 3), material per triangle
    (MAT_*), colour per triangle (albedo / radiance / C_tex / transmittance)."""

    def __init__(self, tris, types, rgb, n_verts):
        self._t = _i32(tris)
        self._ty = _i32(types)
        self._rgb = np.ascontiguousarray(rgb, dtype=np.float32)
        d = RenderScene(int(n_verts), len(self._t), self._t.ctypes.data_as(ip), self._ty.ctypes.data_as(ip),
                        self._rgb.ctypes.data_as(C.POINTER(C.c_float)))
        h = C.c_void_p()
        code = load().sim_render_create(C.byref(d), C.byref(h))
        if code != IPC_OK:
            raise IpcError(code, load().sim_render_last_error().decode())
        self.h = h

    def render(self, x_dev, cam, spp=4, max_depth=2, n_shadow=8, lambda_s=0.8, eps=1e-5, seed=0, out=None,
               stream=None):
        """Linear-RGB frame (height, width, 3) float32 on the device at vertex positions x_dev (n, 3) float64.
        cam: (13 floats eye, fwd, right, up, tan(fov/2)), width, height."""
        import torch
        c, w, h = cam
        c = np.asarray(c, np.float32)
        cm = Camera()
        for k in range(3):
            cm.eye[k], cm.fwd[k], cm.right[k], cm.up[k] = float(c[k]), float(c[3 + k]), float(c[6 + k]), float(c[9 + k])
        cm.tan_half_fov, cm.width, cm.height = float(c[12]), int(w), int(h)
        p = RenderParams(int(spp), int(max_depth), int(n_shadow), float(lambda_s), float(eps), int(seed))
        if out is None:
            out = torch.empty((h, w, 3), dtype=torch.float32, device=x_dev.device)
        st = C.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
        code = load().sim_render_frame(self.h, _ptr(x_dev.contiguous()), C.byref(cm), C.byref(p), _ptr(out), st)
        if code != IPC_OK:
            raise IpcError(code, "sim_render_frame failed")
        return out

    def close(self):
        if getattr(self, "h", None):
            load().sim_render_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def step_many(sims, kin_T_next=None):
    """Advance independent simulators one step each, concurrently (one stream and host thread per scene).

    kin_T_next: list of (n_kin, 3, 4) arrays (None entries for scenes without kinematic bodies); defaults to
    each scene's trajectory.  Returns the list of per-scene stats dicts."""
    n = len(sims)
    handles = (vp * n)(*[s.h for s in sims])
    arrs = []
    ptrs = (dp * n)()
    for i, s in enumerate(sims):
        s._trajectory_joint_targets(s.step_index + 1)
        T = kin_T_next[i] if kin_T_next is not None else (s.scene["kin_T"][s.step_index + 1] if s.nkb else None)
        if T is not None and s.nkb:
            a = _f64(T).reshape(-1)
            arrs.append(a)
            ptrs[i] = a.ctypes.data_as(dp)
        else:
            ptrs[i] = None
    stats = (StepStats * n)()
    status = (C.c_int * n)()
    load().sim_step_many(handles, n, ptrs, stats, status)
    out = []
    for i, s in enumerate(sims):
        if status[i] == IPC_OK:
            s.step_index += 1
        out.append(stats[i].as_dict())
    return out
