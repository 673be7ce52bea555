"""Seeded synthetic inputs for the neural shadow method (input generator only).

The paper's scenes (Bistro, Sponza, ...) and its Falcor rasteriser are not
available, so every input is produced by ray casting a seeded analytic scene:
an infinite ground plane z = 0 plus axis-aligned boxes and spheres, one point
or spherical emitter, a pinhole camera and a single-frustum ("vanilla")
shadow map (Sec. 3.1 lists the buffers; Sec. 1 and suppl. Sec. 5 say the
shadow map is a single frustum that covers the camera's view).

This module holds none of the method's arithmetic: it writes the G-buffer
(world position + view depth, normal), the shadow-map depths, the light's
world-to-clip matrix, and the ray-traced visibility targets.  Both the FP64
oracle and the CUDA path read what it writes.

Scene recipe (all draws from one SplitMix64 stream per seed):
  * objects: sphere or box with probability 1/2; centre ~ U([-1,1]^2 x [0,0.5]);
    size s ~ U[0.05, 0.3] (sphere radius, box half-extent);
  * emitter: centre at distance 3 from the origin, direction uniform on the
    spherical cap of elevation >= 20 degrees; spherical emitters have
    radius r ~ U[0.05, 0.2] (point light: r = 0);
  * camera: C = (0, -2.5, 3) looking at the origin, up +z, vertical fov 36 deg,
    framing the object region so that the view stays (almost entirely) inside
    the emitter frustum, as the paper arranges its camera paths (suppl. Sec. 5),
    and every visible receiver lies within z_far of the emitter;
  * shadow-map frustum: looks at the origin, up +y, fov = 2 asin(2 / |L|),
    near 0.05, far (z_far) 10; texels whose ray meets nothing read z_far.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "raycast.c")
_LIB_PATH = os.path.join(_HERE, "libraycast.so")
_lock = threading.Lock()
_lib = None

Z_FAR = 10.0
Z_NEAR = 0.05
SHADOW_EPS = 1e-4
SM_BOUND_RADIUS = 2.0


def build(force: bool = False) -> str:
    """Compile raycast.c into a shared library next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            lib.sg_gbuffer.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, P, P, P]
            lib.sg_shadowmap.argtypes = [ctypes.c_int, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_double, P]
            lib.sg_hard_visibility.argtypes = [ctypes.c_size_t, P, P, P, P, ctypes.c_int, P, ctypes.c_double, P]
            lib.sg_soft_visibility.argtypes = [ctypes.c_size_t, P, P, P, P, ctypes.c_double, ctypes.c_int, P,
                                               ctypes.c_int, ctypes.c_uint64, ctypes.c_double, P]
            lib.sg_light_depth.argtypes = [ctypes.c_size_t, P, P, ctypes.c_int, P, P]
            lib.sg_trace_one.argtypes = [P, P, ctypes.c_int, P, ctypes.c_int, P]
            lib.sg_trace_one.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------- RNG
class SplitMix64:
    """SplitMix64 (Steele, Lea & Flood, OOPSLA 2014); platform independent."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / 9007199254740992.0))

    def normal(self) -> float:
        u1 = max(self.uniform(), 1e-300)
        u2 = self.uniform()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------- scene
@dataclasses.dataclass
class Scene:
    objects: np.ndarray          # (n, 5) float64: type, cx, cy, cz, s
    light_pos: np.ndarray        # (3,) float64
    light_radius: float          # 0 for a point light
    cam_pos: np.ndarray = dataclasses.field(default_factory=lambda: np.array([0.0, -2.5, 3.0]))
    cam_target: np.ndarray = dataclasses.field(default_factory=lambda: np.array([0.0, 0.0, 0.0]))
    cam_up: np.ndarray = dataclasses.field(default_factory=lambda: np.array([0.0, 0.0, 1.0]))
    cam_fovy_deg: float = 36.0


def random_objects(rng: SplitMix64, n: int) -> np.ndarray:
    obj = np.zeros((n, 5), np.float64)
    for i in range(n):
        obj[i, 0] = 0.0 if rng.uniform() < 0.5 else 1.0
        obj[i, 1] = rng.uniform(-1.0, 1.0)
        obj[i, 2] = rng.uniform(-1.0, 1.0)
        obj[i, 3] = rng.uniform(0.0, 0.5)
        obj[i, 4] = rng.uniform(0.05, 0.3)
    return obj


def random_light_dir(rng: SplitMix64, min_elev_deg: float = 20.0) -> np.ndarray:
    """Uniform direction on the cap of elevation >= min_elev_deg."""
    zmin = math.sin(math.radians(min_elev_deg))
    z = rng.uniform(zmin, 1.0)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    s = math.sqrt(max(0.0, 1.0 - z * z))
    return np.array([s * math.cos(phi), s * math.sin(phi), z])


def random_scene(seed: int, n_obj: int, soft: bool = False, light_dist: float = 3.0) -> Scene:
    rng = SplitMix64(seed)
    obj = random_objects(rng, n_obj)
    L = light_dist * random_light_dir(rng)
    r = rng.uniform(0.05, 0.2) if soft else 0.0
    return Scene(objects=obj, light_pos=L, light_radius=r)


def emitter_size_feature(radius: float) -> float:
    """Emitter-size value r_hat in [0, 4]: 4 = 50 cm diameter (Sec. 3.1.1)."""
    return float(min(max(4.0 * (2.0 * radius) / 0.5, 0.0), 4.0))


def _look_basis(eye, target, up):
    fwd = np.asarray(target, np.float64) - np.asarray(eye, np.float64)
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    return fwd, right, upv


def light_frustum(L: np.ndarray):
    """Light view basis, tan(fov/2) and the FP64 world->clip matrix (row-major)."""
    fwd, right, up = _look_basis(L, np.zeros(3), np.array([0.0, 1.0, 0.0]))
    fov = 2.0 * math.asin(min(1.0, SM_BOUND_RADIUS / float(np.linalg.norm(L))))
    t = math.tan(0.5 * fov)
    V = np.eye(4)
    V[0, :3] = right; V[0, 3] = -right @ L
    V[1, :3] = up;    V[1, 3] = -up @ L
    V[2, :3] = -fwd;  V[2, 3] = fwd @ L
    f = 1.0 / t
    n, fa = Z_NEAR, Z_FAR
    Pm = np.zeros((4, 4))
    Pm[0, 0] = f
    Pm[1, 1] = f
    Pm[2, 2] = (fa + n) / (n - fa)
    Pm[2, 3] = 2.0 * fa * n / (n - fa)
    Pm[3, 2] = -1.0
    return fwd, right, up, t, Pm @ V


@dataclasses.dataclass
class Frame:
    """One view: everything the hot path consumes, as float32 host arrays."""
    H: int
    W: int
    pos4: np.ndarray      # (H, W, 4) float32: world P, w = view depth d
    nrm4: np.ndarray      # (H, W, 4) float32: unit normal, w = 0
    mask: np.ndarray      # (H, W) uint8: 1 where the camera ray hit geometry
    sm: np.ndarray        # (Hs, Ws) float32 emitter-to-occluder distance
    view_proj: np.ndarray  # (4, 4) float32 light world->clip, row-major
    light_pos: np.ndarray  # (3,) float32
    light_radius: float
    r_hat: float
    cam_pos: np.ndarray   # (3,) float32
    z_far: float
    bias: float           # relative depth bias beta (test: z_f <= z + beta z_f)
    tan_half_fov: float
    scene: Scene

    @property
    def Hs(self):
        return self.sm.shape[0]

    @property
    def Ws(self):
        return self.sm.shape[1]


def camera_vector(scene: Scene, H: int, W: int) -> np.ndarray:
    """The eye camera as the GPU generator takes it: eye, forward, right, up,
    tan(fovy / 2), aspect W / H (14 values)."""
    fwd, right, up = _look_basis(scene.cam_pos, scene.cam_target, scene.cam_up)
    th = math.tan(math.radians(scene.cam_fovy_deg) * 0.5)
    return np.concatenate([scene.cam_pos, fwd, right, up, [th, W / H]])


def light_camera_vector(scene: Scene) -> np.ndarray:
    """The light camera as the GPU generator takes it: centre, forward, right,
    up, tan(fov / 2) (13 values)."""
    lf, lr, lu, lt, _ = light_frustum(np.asarray(scene.light_pos, np.float64))
    return np.concatenate([scene.light_pos, lf, lr, lu, [lt]])


def default_bias(tan_half_fov: float, Ws: int) -> float:
    """Relative depth bias beta = two texel angular widths, 2 * (2 tan(fov/2) / Ws).
    The depth test compares z_f <= z + beta * z_f, so the bias grows with the
    receiver distance like the texel footprint does.  A constant world-space
    bias small enough to avoid light leaks (e.g. 2e-3) leaves shadow acne over
    most of the far ground plane at these map resolutions."""
    return 2.0 * (2.0 * tan_half_fov / Ws)


def render_frame(scene: Scene, H: int, W: int, Hs: int, Ws: int, bias: float | None = None) -> Frame:
    lib = _load()
    obj = np.ascontiguousarray(scene.objects, np.float64)
    fwd, right, up = _look_basis(scene.cam_pos, scene.cam_target, scene.cam_up)
    th = math.tan(math.radians(scene.cam_fovy_deg) * 0.5)
    cam = np.concatenate([scene.cam_pos, fwd, right, up, [th, W / H]]).astype(np.float64)
    pos4 = np.empty((H, W, 4), np.float32)
    nrm4 = np.empty((H, W, 4), np.float32)
    mask = np.empty((H, W), np.uint8)
    lib.sg_gbuffer(H, W, _ptr(cam), obj.shape[0], _ptr(obj), _ptr(pos4), _ptr(nrm4), _ptr(mask))
    L = np.asarray(scene.light_pos, np.float64)
    lf, lr, lu, lt, VP = light_frustum(L)
    lcam = np.concatenate([L, lf, lr, lu, [lt]]).astype(np.float64)
    if bias is None:
        bias = default_bias(lt, Ws)
    sm = np.empty((Hs, Ws), np.float32)
    lib.sg_shadowmap(Hs, Ws, _ptr(lcam), obj.shape[0], _ptr(obj), Z_FAR, _ptr(sm))
    return Frame(H=H, W=W, pos4=pos4, nrm4=nrm4, mask=mask, sm=sm,
                 view_proj=VP.astype(np.float32), light_pos=L.astype(np.float32),
                 light_radius=float(scene.light_radius), r_hat=emitter_size_feature(scene.light_radius),
                 cam_pos=np.asarray(scene.cam_pos, np.float32), z_far=Z_FAR, bias=bias,
                 tan_half_fov=lt, scene=scene)


def light_depth_exact(frame: Frame) -> np.ndarray:
    """Distance from the emitter centre to the first hit along the exact ray
    towards each pixel's position (the shadow-map depth at infinite map
    resolution): (H, W) float64."""
    lib = _load()
    obj = np.ascontiguousarray(frame.scene.objects, np.float64)
    L = np.asarray(frame.scene.light_pos, np.float64)
    out = np.empty((frame.H, frame.W), np.float64)
    lib.sg_light_depth(frame.H * frame.W, _ptr(frame.pos4), _ptr(L), obj.shape[0], _ptr(obj), _ptr(out))
    return out


def hard_visibility(frame: Frame, eps: float = SHADOW_EPS) -> np.ndarray:
    """Brute-force shadow rays to the emitter centre: (H, W) uint8, 1 = lit."""
    lib = _load()
    obj = np.ascontiguousarray(frame.scene.objects, np.float64)
    L = np.asarray(frame.scene.light_pos, np.float64)
    vis = np.empty((frame.H, frame.W), np.uint8)
    lib.sg_hard_visibility(frame.H * frame.W, _ptr(frame.pos4), _ptr(frame.nrm4), _ptr(frame.mask),
                           _ptr(L), obj.shape[0], _ptr(obj), eps, _ptr(vis))
    return vis


def soft_visibility(frame: Frame, spp_side: int = 32, seed: int = 7, eps: float = SHADOW_EPS,
                    radius: float | None = None) -> np.ndarray:
    """Monte-Carlo visibility of the spherical emitter (spp_side^2 samples/pixel)."""
    lib = _load()
    obj = np.ascontiguousarray(frame.scene.objects, np.float64)
    L = np.asarray(frame.scene.light_pos, np.float64)
    r = frame.light_radius if radius is None else radius
    vis = np.empty((frame.H, frame.W), np.float32)
    lib.sg_soft_visibility(frame.H * frame.W, _ptr(frame.pos4), _ptr(frame.nrm4), _ptr(frame.mask),
                           _ptr(L), float(r), obj.shape[0], _ptr(obj), spp_side,
                           ctypes.c_uint64(seed), eps, _ptr(vis))
    return vis


def trace_one(o, d, objects, with_plane=True):
    """Nearest hit (t, normal) along one unit ray, t = -1 when nothing is hit."""
    lib = _load()
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    obj = np.ascontiguousarray(np.asarray(objects, np.float64).reshape(-1, 5))
    n = np.zeros(3, np.float64)
    t = lib.sg_trace_one(_ptr(o), _ptr(d), obj.shape[0], _ptr(obj) if obj.size else None,
                         1 if with_plane else 0, _ptr(n))
    return t, n


# --------------------------------------------------------------------------- workloads
def hard_frame(H: int, W: int, Hs: int, Ws: int, n_obj: int, seed: int) -> Frame:
    """Hard shadow frame: point light (r_hat = 0)."""
    return render_frame(random_scene(seed, n_obj, soft=False), H, W, Hs, Ws)


def soft_frame(H: int, W: int, Hs: int, Ws: int, n_obj: int, seed: int) -> Frame:
    """Soft shadow frame: spherical emitter of radius U[0.05, 0.2]."""
    return render_frame(random_scene(seed, n_obj, soft=True), H, W, Hs, Ws)


def temporal_sequence(H: int, W: int, Hs: int, Ws: int, n_obj: int, seed: int, n_frames: int = 8,
                      orbit_deg: float = 2.0, n_moving: int = 4, speed: float = 0.01):
    """Soft-shadow sequence: the emitter orbits the z axis by orbit_deg per frame
    at fixed elevation; n_moving seeded objects translate speed units per frame
    along a seeded xy direction."""
    base = random_scene(seed, n_obj, soft=True)
    rng = SplitMix64(seed ^ 0x5EED)
    dirs = []
    for _ in range(min(n_moving, n_obj)):
        a = rng.uniform(0.0, 2.0 * math.pi)
        dirs.append((math.cos(a), math.sin(a)))
    frames = []
    for t in range(n_frames):
        obj = base.objects.copy()
        for k, (dx, dy) in enumerate(dirs):
            obj[k, 1] += speed * t * dx
            obj[k, 2] += speed * t * dy
        ang = math.radians(orbit_deg * t)
        c, s = math.cos(ang), math.sin(ang)
        L = base.light_pos
        Lt = np.array([c * L[0] - s * L[1], s * L[0] + c * L[1], L[2]])
        sc = Scene(objects=obj, light_pos=Lt, light_radius=base.light_radius)
        frames.append(render_frame(sc, H, W, Hs, Ws))
    return frames


def perturbed(scene: Scene, rng: SplitMix64) -> Scene:
    """Jitter the emitter by a radius 0.005|L| + 0.25 r and the camera by
    0.005|C| (uniform in a ball): the training-time perturbations whose size
    grows with the distance to the scene and the emitter size (Sec. 3.3)."""
    def ball(radius):
        while True:
            v = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-1, 1)])
            if v @ v <= 1.0:
                return radius * v
    L = np.asarray(scene.light_pos, np.float64)
    C = np.asarray(scene.cam_pos, np.float64)
    rl = 0.005 * np.linalg.norm(L) + 0.25 * scene.light_radius
    rc = 0.005 * np.linalg.norm(C)
    return dataclasses.replace(scene, light_pos=L + ball(rl), cam_pos=C + ball(rc),
                               cam_target=np.asarray(scene.cam_target) + 0.0)


TRAINED_WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights_trained_3level.npy")


def trained_weights() -> np.ndarray:
    """Seeded trained weights of the 3-level network (canonical order, float32):
    one network for hard and soft shadows, trained on this module's ray-cast
    targets by the oracle's training step (`python -m oracle.train_weights`,
    which documents the recipe).  An input like the scenes, not an expected
    value."""
    if not os.path.exists(TRAINED_WEIGHTS):
        raise FileNotFoundError(f"{TRAINED_WEIGHTS} is missing (python -m oracle.train_weights writes it)")
    return np.load(TRAINED_WEIGHTS).astype(np.float32)


TRAINED_WEIGHTS_S2D = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights_trained_s2d.npy")


def trained_weights_s2d() -> np.ndarray:
    """Seeded trained weights of the space-to-depth network (Sec. 3.5), same
    recipe as trained_weights (`python -m oracle.train_weights --topology s2d`)."""
    if not os.path.exists(TRAINED_WEIGHTS_S2D):
        raise FileNotFoundError(f"{TRAINED_WEIGHTS_S2D} is missing "
                                "(python -m oracle.train_weights --topology s2d writes it)")
    return np.load(TRAINED_WEIGHTS_S2D).astype(np.float32)


def he_init_weights(seed: int, layers) -> np.ndarray:
    """Seeded He-normal weights (std sqrt(2 / fan_in)), zero biases, flattened
    in the canonical order: for each layer OIHW weights then its bias."""
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = []
    for (_, cin, cout, k) in layers:
        std = math.sqrt(2.0 / (cin * k * k))
        parts.append(rng.standard_normal(cout * cin * k * k) * std)
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float64)
