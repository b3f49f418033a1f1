"""ctypes binding of include/rsi.h (argument marshalling only).

Every numerical step runs in librsi.so's CUDA kernels; this module only
allocates device buffers with PyTorch, passes pointers, sizes and the current
stream, and raises on a non-zero status.  There is no fallback: if the
library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librsi.so")


def _lib_path() -> str:
    from paper_2408_06765_gb300 import build as _build  # the same rule as the build (RSI_BUILD_DEFINES)
    return os.path.join(_build.build_dir(), "librsi.so")
_lock = threading.Lock()
_lib = None

# --- constants mirrored from include/rsi.h -----------------------------------
RSI_OK = 0
PF = dict(IDX=0, SU=1, SV=2, X=3, Y=4, Z=5, NX=6, NY=7, NZ=8, W=9,
          XH=10, XL=11, YH=12, YL=13, ZH=14, ZL=15)
PF_DTYPE = {**{k: torch.int32 for k in ("IDX", "SU", "SV")},
            **{k: torch.float64 for k in ("X", "Y", "Z", "NX", "NY", "NZ", "W")},
            **{k: torch.float32 for k in ("XH", "XL", "YH", "YL", "ZH", "ZL")}}
SURF = {"disk": 0, "rect": 1, "cyl": 2, "cap": 3}
SEQ = {"sobol": 0, "halton": 1}
STAGE_PISTON, STAGE_RSI = 0, 1
PREC = {"fp64": 0, "fp32c": 1}
NORMALS_Z, NORMALS_POINTS, NORMALS_NEG_Z, NORMALS_POINTS_NEG = 0, 1, 2, 3
TMODE = {"global": 0, "local": 1}
IMG = {"c128": 0, "c64": 1, "abs32": 2}

SYMBOLS = ["rsi_version", "rsi_last_error", "rsi_sync_status", "rsi_points_bytes",
           "rsi_points_offset", "rsi_make_qmc_points", "rsi_grid_points", "rsi_points_slice",
           "rsi_stage_workspace_bytes", "rsi_propagate_stage", "rsi_propagate_stage_noalloc",
           "rsi_interface_transmit",
           "rsi_interface_reflect", "rsi_field_image", "rsi_field_image_sum", "rsi_launch_count",
           "rsi_raytrace_workspace_bytes", "rsi_raytrace_field", "rsi_stage_multi_workspace_bytes",
           "rsi_propagate_stage_multi", "rsi_stage_multi_shared_harmonic", "rsi_timing_enable", "rsi_timing_read",
           "rsi_ubench", "rsi_autotune_stage", "rsi_batch_create", "rsi_batch_run",
           "rsi_batch_destroy", "rsi_nn_features", "rsi_nn_gemm", "rsi_nn_transpose", "rsi_nn_loss",
           "rsi_nn_colsum", "rsi_nn_adam", "rsi_nn_adam_dev", "rsi_nn_cast_bf16", "rsi_nn_carrier", "rsi_nn_gemm_carrier", "rsi_nn_carrier_coeffs",
           "rsi_selftest_wait_timeout", "rsi_nn_param_elems", "rsi_nn_param_offset", "rsi_nn_act_bytes",
           "rsi_nn_rows", "rsi_nn_forward", "rsi_nn_backward", "rsi_nn_adam_step", "rsi_nn_targets",
           "rsi_nn_infer"]
NN_EPI = {"f32": 0, "bias_silu": 1, "dsilu": 2}
NN_ENGINE = {"mma_sync": 0, "tcgen05": 1}
UB = {"ffma": 0, "rsqrt": 1, "sin": 2, "dfma": 3}


class Surface(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("scramble", ctypes.c_int32),
                ("centre", ctypes.c_double * 3), ("tilt", ctypes.c_double),
                ("a", ctypes.c_double), ("wx", ctypes.c_double), ("wy", ctypes.c_double),
                ("R", ctypes.c_double), ("sequence", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("apod", ctypes.c_double)]


class Grid(ctypes.Structure):
    _fields_ = [("x0", ctypes.c_double), ("x1", ctypes.c_double), ("z0", ctypes.c_double),
                ("z1", ctypes.c_double), ("y", ctypes.c_double), ("nx", ctypes.c_int32),
                ("nz", ctypes.c_int32)]


class Stage(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("precision", ctypes.c_int32), ("k", ctypes.c_double),
                ("v0", ctypes.c_double), ("normals", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("tpt", ctypes.c_int32), ("splits", ctypes.c_int32), ("variant", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Interface(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("reserved", ctypes.c_int32), ("rho1", ctypes.c_double),
                ("c1", ctypes.c_double), ("rho2", ctypes.c_double), ("c2", ctypes.c_double),
                ("snell_C", ctypes.c_double)]


class Raytrace(ctypes.Structure):
    _fields_ = [("k1", ctypes.c_double), ("k2", ctypes.c_double), ("rho1", ctypes.c_double),
                ("c1", ctypes.c_double), ("rho2", ctypes.c_double), ("c2", ctypes.c_double),
                ("z_interface", ctypes.c_double), ("v0", ctypes.c_double), ("tile", ctypes.c_int32),
                ("splits", ctypes.c_int32), ("newton", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class NNNet(ctypes.Structure):
    _fields_ = [("n_freq", ctypes.c_int32), ("width", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("rows", ctypes.c_int32), ("engine", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("c1", ctypes.c_double), ("c2", ctypes.c_double), ("a", ctypes.c_double),
                ("box_lo", ctypes.c_double * 4), ("box_hi", ctypes.c_double * 4), ("window", Grid),
                ("fmat", ctypes.c_void_p)]


class BatchInstance(ctypes.Structure):
    _fields_ = [("piston", Surface), ("iface", Surface), ("n_piston", ctypes.c_int64),
                ("n_iface", ctypes.c_int64), ("piston_set", ctypes.c_uint32),
                ("iface_set", ctypes.c_uint32), ("transmit", Interface), ("k1", ctypes.c_double),
                ("k2", ctypes.c_double), ("v0", ctypes.c_double), ("grid", Grid)]


class RSIError(RuntimeError):
    def __init__(self, what: str, code: int, msg: str):
        super().__init__(f"{what} failed ({code}): {msg}")
        self.code = code


def load(path: str | None = None):
    """Load librsi.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _lib_path()
        if not os.path.exists(p):
            raise RuntimeError(f"librsi.so not built ({p}); run paper_2408_06765_gb300.build")
        L = ctypes.CDLL(p)
        vp, i32, i64, u32, u64, sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t)
        L.rsi_version.restype = ctypes.c_int
        L.rsi_last_error.restype = ctypes.c_char_p
        L.rsi_sync_status.argtypes = [vp]
        L.rsi_points_bytes.restype = sz
        L.rsi_points_bytes.argtypes = [i64]
        L.rsi_points_offset.restype = i64
        L.rsi_points_offset.argtypes = [i32, i64]
        L.rsi_make_qmc_points.argtypes = [ctypes.POINTER(Surface), u64, u32, i64, vp, sz, vp]
        L.rsi_grid_points.argtypes = [ctypes.POINTER(Grid), vp, sz, vp]
        L.rsi_points_slice.argtypes = [vp, i64, i64, i64, vp, sz, vp]
        L.rsi_stage_workspace_bytes.restype = sz
        L.rsi_stage_workspace_bytes.argtypes = [ctypes.POINTER(Stage), i64, i64]
        L.rsi_propagate_stage.argtypes = [ctypes.POINTER(Stage), vp, i64, vp, vp, i64, vp, vp, sz, vp]
        L.rsi_propagate_stage_noalloc.argtypes = [ctypes.POINTER(Stage), vp, i64, vp, vp, i64, vp, vp]
        L.rsi_interface_transmit.argtypes = [ctypes.POINTER(Interface), vp, i64, vp, vp, vp]
        L.rsi_field_image.argtypes = [ctypes.POINTER(Grid), vp, ctypes.c_double, ctypes.c_double,
                                      i32, vp, vp]
        L.rsi_interface_reflect.argtypes = [ctypes.POINTER(Interface), vp, i64, vp, vp, vp]
        L.rsi_stage_multi_workspace_bytes.restype = sz
        L.rsi_stage_multi_workspace_bytes.argtypes = [ctypes.POINTER(Stage), i32, vp, i64, i64]
        L.rsi_stage_multi_shared_harmonic.argtypes = [ctypes.POINTER(Stage), i32, vp]
        L.rsi_propagate_stage_multi.argtypes = [ctypes.POINTER(Stage), i32, vp, vp, i64, vp, vp, i64, vp, vp, sz,
                                                vp]
        L.rsi_raytrace_workspace_bytes.restype = sz
        L.rsi_raytrace_workspace_bytes.argtypes = [ctypes.POINTER(Raytrace), i64, i64]
        L.rsi_raytrace_field.argtypes = [ctypes.POINTER(Raytrace), vp, i64, vp, i64, vp, vp, sz, vp]
        L.rsi_field_image_sum.argtypes = [ctypes.POINTER(Grid), vp, vp, ctypes.c_double, ctypes.c_double,
                                          i32, vp, vp]
        L.rsi_launch_count.restype = u64
        L.rsi_timing_enable.argtypes = [i32]
        L.rsi_timing_read.argtypes = [i32, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]
        L.rsi_ubench.argtypes = [i32, i32, i32, vp, vp]
        L.rsi_autotune_stage.argtypes = [ctypes.POINTER(Stage), vp, i64, vp, vp, i64, vp, vp, sz, vp,
                                         ctypes.POINTER(Stage)]
        L.rsi_batch_create.argtypes = [ctypes.POINTER(BatchInstance), i32, u64, ctypes.POINTER(Stage),
                                       ctypes.POINTER(vp), ctypes.POINTER(sz), ctypes.POINTER(sz)]
        L.rsi_batch_run.argtypes = [vp, vp, sz, vp, vp]
        L.rsi_batch_destroy.argtypes = [vp]
        f32, f64 = ctypes.c_float, ctypes.c_double
        L.rsi_nn_features.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp, vp]
        L.rsi_nn_gemm.argtypes = [i32, i32, i32, vp, vp, i32, i32, i32, vp, vp, vp, vp, i32, vp, vp]
        L.rsi_nn_transpose.argtypes = [vp, i32, i32, vp, vp]
        L.rsi_nn_loss.argtypes = [vp, vp, i64, f32, vp, vp, i32, vp, vp]
        L.rsi_nn_colsum.argtypes = [vp, i32, i32, vp, vp]
        L.rsi_nn_adam.argtypes = [vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp, vp]
        L.rsi_nn_adam_dev.argtypes = [vp, vp, vp, vp, i64, vp, f32, f32, f32, vp, vp]
        L.rsi_nn_carrier_coeffs.argtypes = [vp, i32, ctypes.c_double, ctypes.c_double, vp, vp, vp]
        L.rsi_nn_gemm_carrier.argtypes = [vp, vp, i32, i32, i32, vp, vp, ctypes.POINTER(Grid), i32, f32, vp, vp,
                                          vp]
        L.rsi_nn_cast_bf16.argtypes = [vp, i64, vp, vp]
        L.rsi_nn_carrier.argtypes = [vp, i32, ctypes.POINTER(Grid), i32, ctypes.c_float, vp, vp, vp]
        L.rsi_selftest_wait_timeout.argtypes = [i64, vp]
        pn = ctypes.POINTER(NNNet)
        L.rsi_nn_param_elems.restype = i64
        L.rsi_nn_param_elems.argtypes = [pn]
        L.rsi_nn_param_offset.restype = i64
        L.rsi_nn_param_offset.argtypes = [pn, i32, i32]
        L.rsi_nn_act_bytes.restype = sz
        L.rsi_nn_act_bytes.argtypes = [pn]
        L.rsi_nn_rows.argtypes = [pn, vp, i64, i32, u64, vp, i64, vp, vp, vp, sz, vp]
        L.rsi_nn_forward.argtypes = [pn, vp, vp, vp, sz, vp, vp]
        L.rsi_nn_backward.argtypes = [pn, vp, vp, vp, sz, vp, vp, vp]
        L.rsi_nn_adam_step.argtypes = [pn, vp, vp, vp, vp, vp, vp, f32, f32, f32, vp]
        L.rsi_nn_targets.argtypes = [pn, vp, i32, vp, vp, vp, vp, vp, vp, vp]
        L.rsi_nn_infer.argtypes = [pn, vp, vp, vp, i32, vp, sz, vp, vp, vp]
        _lib = L
        return L


def _check(rc: int, what: str):
    if rc != RSI_OK:
        raise RSIError(what, rc, load().rsi_last_error().decode(errors="replace"))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


# ---------------------------------------------------------------------------
# point sets
# ---------------------------------------------------------------------------
class Points:
    """A point set: one device buffer in the layout of include/rsi.h."""

    def __init__(self, n: int, device="cuda"):
        L = load()
        self.n = int(n)
        self.nbytes = int(L.rsi_points_bytes(self.n))
        self.buf = torch.empty(self.nbytes, dtype=torch.uint8, device=device)
        if self.buf.data_ptr() % 256:
            raise RuntimeError("point buffer is not 256-byte aligned")

    def field(self, name: str) -> torch.Tensor:
        """Typed view of one field (IDX/SU/SV are uint32 stored as int32)."""
        off = int(load().rsi_points_offset(PF[name], self.n))
        dt = PF_DTYPE[name]
        nb = self.n * torch.empty(0, dtype=dt).element_size()
        return self.buf[off:off + nb].view(dt)

    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr())


def surface_struct(surf: dict, scramble: bool = True) -> Surface:
    s = Surface()
    s.kind = SURF[surf["kind"]]
    s.scramble = 1 if scramble else 0
    for i, v in enumerate(surf.get("centre", (0.0, 0.0, 0.0))):
        s.centre[i] = float(v)
    s.tilt = float(surf.get("tilt", 0.0))
    s.a = float(surf.get("a", 0.0))
    s.wx = float(surf.get("wx", 0.0))
    s.wy = float(surf.get("wy", 0.0))
    s.R = float(surf.get("R", 0.0))
    s.sequence = SEQ[surf.get("sequence", "sobol")]
    if s.sequence == SEQ["halton"]:
        s.scramble = 0
    s.apod = float(surf.get("apod", 0.0))
    return s


def make_qmc_points(surf: dict, seed: int, set_id: int, n: int, scramble: bool = True,
                    device="cuda", stream=None, out: Points | None = None) -> Points:
    pts = out if out is not None else Points(n, device)
    s = surface_struct(surf, scramble)
    _check(load().rsi_make_qmc_points(ctypes.byref(s), int(seed) & (2**64 - 1), int(set_id), int(n),
                                      pts.ptr(), pts.nbytes, _stream(stream)), "rsi_make_qmc_points")
    return pts


def grid_struct(g: dict) -> Grid:
    G = Grid()
    G.x0, G.x1, G.z0, G.z1 = (float(g[k]) for k in ("x0", "x1", "z0", "z1"))
    G.y = float(g.get("y", 0.0))
    G.nx, G.nz = int(g["nx"]), int(g["nz"])
    return G


def grid_points(g: dict, device="cuda", stream=None, out: Points | None = None) -> Points:
    G = grid_struct(g)
    pts = out if out is not None else Points(G.nx * G.nz, device)
    _check(load().rsi_grid_points(ctypes.byref(G), pts.ptr(), pts.nbytes, _stream(stream)),
           "rsi_grid_points")
    return pts


def points_slice(pts: Points, first: int, count: int, stream=None, out: Points | None = None) -> Points:
    """Slots [first, first + count) of a point set as a point set of its own."""
    sub = out if out is not None else Points(count, pts.buf.device)
    _check(load().rsi_points_slice(pts.ptr(), pts.n, int(first), int(count), sub.ptr(), sub.nbytes,
                                   _stream(stream)), "rsi_points_slice")
    return sub


# ---------------------------------------------------------------------------
# stages
# ---------------------------------------------------------------------------
def stage_struct(kind: int, precision: str, k: float, v0: float = 1.0, normals: int = NORMALS_Z,
                 tile: int = 0, tpt: int = 0, splits: int = 0, variant: int = 0) -> Stage:
    st = Stage()
    st.kind, st.precision = int(kind), PREC[precision]
    st.k, st.v0 = float(k), float(v0)
    st.normals, st.tile, st.tpt, st.splits, st.variant = (int(normals), int(tile), int(tpt),
                                                          int(splits), int(variant))
    return st


def workspace_bytes(st: Stage, n_src: int, n_tgt: int) -> int:
    nb = int(load().rsi_stage_workspace_bytes(ctypes.byref(st), int(n_src), int(n_tgt)))
    if nb == 0:
        raise RSIError("rsi_stage_workspace_bytes", -1, load().rsi_last_error().decode())
    return nb


class Workspace:
    """Grow-only device scratch buffer shared by successive stage calls."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf


def propagate_stage(st: Stage, src: Points, sigma, tgt: Points, out=None,
                    workspace: Workspace | None = None, stream=None) -> torch.Tensor:
    """Field at `tgt` (complex128 [n_tgt], slot order) from sources `src`."""
    if out is None:
        out = torch.empty(tgt.n, dtype=torch.complex128, device=tgt.buf.device)
    ws = (workspace or Workspace(tgt.buf.device)).get(workspace_bytes(st, src.n, tgt.n))
    _check(load().rsi_propagate_stage(ctypes.byref(st), src.ptr(), src.n, _ptr(sigma), tgt.ptr(),
                                      tgt.n, _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
           "rsi_propagate_stage")
    return out


def propagate_stage_multi(st: Stage, ks, src: Points, sigma, tgt: Points, out=None,
                          workspace: Workspace | None = None, stream=None) -> torch.Tensor:
    """nf frequencies of one stage on shared points (rsi_propagate_stage_multi):
    sigma complex [nf, n_src] (RSI) or None, returns complex [nf, n_tgt]."""
    L = load()
    nf = len(ks)
    kd = (ctypes.c_double * nf)(*[float(k) for k in ks])
    if out is None:
        out = torch.empty((nf, tgt.n), dtype=torch.complex128, device=tgt.buf.device)
    nb = int(L.rsi_stage_multi_workspace_bytes(ctypes.byref(st), nf, kd, src.n, tgt.n))
    if nb == 0:
        raise RSIError("rsi_stage_multi_workspace_bytes", -1, L.rsi_last_error().decode(errors="replace"))
    ws = (workspace or Workspace(tgt.buf.device)).get(nb)
    _check(L.rsi_propagate_stage_multi(ctypes.byref(st), nf, kd, src.ptr(), src.n, _ptr(sigma), tgt.ptr(), tgt.n,
                                       _ptr(out), _ptr(ws), nb, _stream(stream)), "rsi_propagate_stage_multi")
    return out


def stage_multi_shared_harmonic(st: Stage, ks) -> bool:
    """Whether rsi_propagate_stage_multi forms one of these frequencies from
    another by the double angle (rsi_stage_multi_shared_harmonic)."""
    kd = (ctypes.c_double * len(ks))(*[float(k) for k in ks])
    rc = int(load().rsi_stage_multi_shared_harmonic(ctypes.byref(st), len(ks), kd))
    if rc < 0:
        _check(rc, "rsi_stage_multi_shared_harmonic")
    return rc == 1


def interface_struct(m_in: dict, m_out: dict, snell_C: float, mode: str = "global") -> Interface:
    it = Interface()
    it.mode = TMODE[mode]
    it.rho1, it.c1 = float(m_in["rho"]), float(m_in["c"])
    it.rho2, it.c2 = float(m_out["rho"]), float(m_out["c"])
    it.snell_C = float(snell_C)
    return it


def interface_transmit(pts: Points, phi, m_in: dict, m_out: dict, snell_C: float,
                       mode: str = "global", out=None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty_like(phi)
    it = interface_struct(m_in, m_out, snell_C, mode)
    _check(load().rsi_interface_transmit(ctypes.byref(it), pts.ptr(), pts.n, _ptr(phi), _ptr(out),
                                         _stream(stream)), "rsi_interface_transmit")
    return out


def interface_reflect(pts: Points, phi, m_in: dict, m_out: dict, snell_C: float,
                      mode: str = "global", out=None, stream=None) -> torch.Tensor:
    """sigma_r = R12 phi: the reflected field's source density (rsi_interface_reflect)."""
    if out is None:
        out = torch.empty_like(phi)
    it = interface_struct(m_in, m_out, snell_C, mode)
    _check(load().rsi_interface_reflect(ctypes.byref(it), pts.ptr(), pts.n, _ptr(phi), _ptr(out),
                                        _stream(stream)), "rsi_interface_reflect")
    return out


def field_image(g: dict, field, k: float, v0: float = 1.0, fmt: str = "c128", out=None,
                stream=None, field_b=None) -> torch.Tensor:
    """(k / v0) (field + field_b) on the grid, [nz][nx]; field_b optional."""
    G = grid_struct(g)
    if out is None:
        dt = {"c128": torch.complex128, "c64": torch.complex64, "abs32": torch.float32}[fmt]
        out = torch.empty((G.nz, G.nx), dtype=dt, device=field.device)
    _check(load().rsi_field_image_sum(ctypes.byref(G), _ptr(field), _ptr(field_b), float(k), float(v0),
                                      IMG[fmt], _ptr(out), _stream(stream)), "rsi_field_image_sum")
    return out


def autotune_stage(st: Stage, src: Points, sigma, tgt: Points, out=None,
                   workspace: Workspace | None = None, max_workspace: int = 1 << 30,
                   stream=None) -> Stage:
    """Fastest FP32C launch shape for this stage (see rsi_autotune_stage)."""
    if out is None:
        out = torch.empty(tgt.n, dtype=torch.complex128, device=tgt.buf.device)
    base = workspace_bytes(st, src.n, tgt.n)
    ws = (workspace or Workspace(tgt.buf.device)).get(max(base, min(max_workspace, 8 * base)))
    best = Stage()
    _check(load().rsi_autotune_stage(ctypes.byref(st), src.ptr(), src.n, _ptr(sigma), tgt.ptr(), tgt.n,
                                     _ptr(out), _ptr(ws), ws.numel(), _stream(stream),
                                     ctypes.byref(best)), "rsi_autotune_stage")
    return best


def sync_status(stream=None):
    _check(load().rsi_sync_status(_stream(stream)), "rsi_sync_status")


def launch_count() -> int:
    """Kernels this library has enqueued in this process."""
    return int(load().rsi_launch_count())


def timing_enable(on: bool = True):
    _check(load().rsi_timing_enable(1 if on else 0), "rsi_timing_enable")


def timing_read(kind: int):
    """(total ms, launches, pairs) of the main stage kernels of `kind` since enable."""
    ms, n, pr = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    _check(load().rsi_timing_read(int(kind), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(pr)),
           "rsi_timing_read")
    return ms.value, n.value, pr.value


def ubench(kind: str, blocks: int, iters: int, sink, stream=None):
    _check(load().rsi_ubench(UB[kind], int(blocks), int(iters), _ptr(sink), _stream(stream)),
           "rsi_ubench")


# ---------------------------------------------------------------------------
# the stage chain of a workload description (paper_2408_06765_gb300.workloads)
# ---------------------------------------------------------------------------
def wavenumber(freq: float, c: float) -> float:
    return 2.0 * math.pi * float(freq) / float(c)


def snell_invariant(cfg: dict) -> float:
    return math.sin(float(cfg["piston"].get("tilt", 0.0))) / float(cfg["media"][0]["c"])


class ChainResult:
    def __init__(self, image, field, ifaces):
        self.image = image    # complex [nz][nx], k phi / v0 (or None)
        self.field = field    # complex128 field at the targets (slot order)
        self.ifaces = ifaces  # [(Points, phi on the points)] when kept


def run_chain(cfg: dict, precision: str | None = None, targets: Points | None = None,
              keep: bool = False, fmt: str = "c128", workspace: Workspace | None = None,
              stage_opts: dict | None = None, stream=None, device="cuda") -> ChainResult:
    """piston -> interfaces -> targets (default: the image grid) on the GPU."""
    prec = precision or cfg.get("precision", "fp32c")
    opts = stage_opts or {}
    ws = workspace or Workspace(device)
    seed = int(cfg.get("seed", 0))
    freq, v0 = float(cfg["freq"]), float(cfg.get("v0", 1.0))
    media = cfg["media"]
    C = snell_invariant(cfg)
    mode = cfg.get("tmode", "global")
    pc = cfg["piston"]
    piston = make_qmc_points(dict({"kind": "disk"}, **pc), seed, int(pc.get("set_id", 0)), int(pc["n"]),
                             device=device, stream=stream)
    ifaces = [make_qmc_points(it, seed, int(it["set_id"]), int(it["n"]), device=device, stream=stream)
              for it in cfg["interfaces"]]
    use_grid = targets is None
    if use_grid:
        targets = grid_points(cfg["grid"], device=device, stream=stream)
    kept = []
    first_tgt = ifaces[0] if ifaces else targets
    st = stage_struct(STAGE_PISTON, prec, wavenumber(freq, media[0]["c"]), v0, **opts)
    phi = propagate_stage(st, piston, None, first_tgt, workspace=ws, stream=stream)
    for s, pts in enumerate(ifaces):
        if keep:
            kept.append((pts, phi))
        sigma = interface_transmit(pts, phi, media[s], media[s + 1], C, mode, stream=stream)
        nxt = ifaces[s + 1] if s + 1 < len(ifaces) else targets
        normals = NORMALS_POINTS if cfg["interfaces"][s]["kind"] != "rect" else NORMALS_Z
        st = stage_struct(STAGE_RSI, prec, wavenumber(freq, media[s + 1]["c"]), 1.0, normals, **opts)
        phi = propagate_stage(st, pts, sigma, nxt, workspace=ws, stream=stream)
    image = None
    if use_grid:
        k_last = wavenumber(freq, media[len(ifaces)]["c"])
        image = field_image(cfg["grid"], phi, k_last, v0, fmt, stream=stream)
    return ChainResult(image, phi, kept)


TIMING_RAYTRACE = 2


def raytrace_struct(cfg: dict, tile: int = 0, splits: int = 0, newton: int = 0) -> Raytrace:
    m = cfg["media"]
    f = float(cfg["freq"])
    return Raytrace(wavenumber(f, m[0]["c"]), wavenumber(f, m[1]["c"]), float(m[0]["rho"]), float(m[0]["c"]),
                    float(m[1]["rho"]), float(m[1]["c"]), float(cfg["interfaces"][0]["centre"][2]),
                    float(cfg.get("v0", 1.0)), int(tile), int(splits), int(newton), 0)


def raytrace_field(rt: Raytrace, src: Points, tgt: Points, out=None, workspace: Workspace | None = None,
                   stream=None) -> torch.Tensor:
    """Eq. transmitted_ray_tracing from transducer points onto targets in medium 2."""
    L = load()
    if out is None:
        out = torch.empty(tgt.n, dtype=torch.complex128, device=tgt.buf.device)
    nb = int(L.rsi_raytrace_workspace_bytes(ctypes.byref(rt), src.n, tgt.n))
    if nb == 0:
        raise RSIError("rsi_raytrace_workspace_bytes", -1, L.rsi_last_error().decode(errors="replace"))
    ws = (workspace or Workspace(tgt.buf.device)).get(nb)
    _check(L.rsi_raytrace_field(ctypes.byref(rt), src.ptr(), src.n, tgt.ptr(), tgt.n, _ptr(out), _ptr(ws), nb,
                                _stream(stream)), "rsi_raytrace_field")
    return out


def run_raytrace(cfg: dict, fmt: str = "c128", workspace: Workspace | None = None, stream=None,
                 device="cuda", **shape) -> torch.Tensor:
    """Image k2 phi_t / v0 of the ray-tracing model (Sec. 2.2) on cfg["grid"]
    (medium 2, below the plane interface at the interface centre's z)."""
    seed = int(cfg.get("seed", 0))
    pc = cfg["piston"]
    piston = make_qmc_points(dict({"kind": "disk"}, **pc), seed, int(pc.get("set_id", 0)), int(pc["n"]),
                             device=device, stream=stream)
    tgt = grid_points(cfg["grid"], device=device, stream=stream)
    rt = raytrace_struct(cfg, **shape)
    phi = raytrace_field(rt, piston, tgt, workspace=workspace, stream=stream)
    return field_image(cfg["grid"], phi, rt.k2, float(cfg.get("v0", 1.0)), fmt, stream=stream)


class TwoMediumResult:
    def __init__(self, image, parts):
        self.image = image  # [nz_w + nz_s][nx], medium-1 rows first
        self.parts = parts  # dict of the fields on the interface and the two windows


def run_two_medium(cfg: dict, precision: str | None = None, fmt: str = "c128",
                   workspace: Workspace | None = None, stage_opts: dict | None = None, stream=None,
                   device="cuda") -> TwoMediumResult:
    """Both media of a one-interface workload (Fig. rayleigh-sommerfeld_integral):
    incident + reflected field in the medium-1 window cfg["grid_water"],
    transmitted field in the medium-2 window cfg["grid_solid"], written into
    one image (medium-1 rows first)."""
    prec = precision or cfg.get("precision", "fp32c")
    opts = stage_opts or {}
    ws = workspace or Workspace(device)
    seed = int(cfg.get("seed", 0))
    freq, v0 = float(cfg["freq"]), float(cfg.get("v0", 1.0))
    m = cfg["media"]
    C = snell_invariant(cfg)
    mode = cfg.get("tmode", "global")
    k1, k2 = wavenumber(freq, m[0]["c"]), wavenumber(freq, m[1]["c"])
    pc, it = cfg["piston"], cfg["interfaces"][0]
    piston = make_qmc_points(dict({"kind": "disk"}, **pc), seed, int(pc.get("set_id", 0)), int(pc["n"]),
                             device=device, stream=stream)
    iface = make_qmc_points(it, seed, int(it["set_id"]), int(it["n"]), device=device, stream=stream)
    gw_cfg, gs_cfg = cfg["grid_water"], cfg["grid_solid"]
    gw = grid_points(gw_cfg, device=device, stream=stream)
    gs = grid_points(gs_cfg, device=device, stream=stream)
    flat = it["kind"] == "rect"
    st1 = stage_struct(STAGE_PISTON, prec, k1, v0, **opts)
    phi_if = propagate_stage(st1, piston, None, iface, workspace=ws, stream=stream)
    phi_inc = propagate_stage(st1, piston, None, gw, workspace=ws, stream=stream)
    sig_r = interface_reflect(iface, phi_if, m[0], m[1], C, mode, stream=stream)
    st_r = stage_struct(STAGE_RSI, prec, k1, 1.0, NORMALS_NEG_Z if flat else NORMALS_POINTS_NEG, **opts)
    phi_ref = propagate_stage(st_r, iface, sig_r, gw, workspace=ws, stream=stream)
    sig_t = interface_transmit(iface, phi_if, m[0], m[1], C, mode, stream=stream)
    st_t = stage_struct(STAGE_RSI, prec, k2, 1.0, NORMALS_Z if flat else NORMALS_POINTS, **opts)
    phi_tr = propagate_stage(st_t, iface, sig_t, gs, workspace=ws, stream=stream)
    dt = {"c128": torch.complex128, "c64": torch.complex64, "abs32": torch.float32}[fmt]
    nw, ns = int(gw_cfg["nz"]), int(gs_cfg["nz"])
    image = torch.empty((nw + ns, int(gw_cfg["nx"])), dtype=dt, device=device)
    field_image(gw_cfg, phi_inc, k1, v0, fmt, out=image[:nw], stream=stream, field_b=phi_ref)
    field_image(gs_cfg, phi_tr, k2, v0, fmt, out=image[nw:], stream=stream)
    parts = {"interface": phi_if, "incident": phi_inc, "reflected": phi_ref, "transmitted": phi_tr}
    return TwoMediumResult(image, parts)


def two_medium_pairs(cfg: dict) -> int:
    """Pair terms of run_two_medium: piston -> interface, piston -> medium-1
    window, interface -> medium-1 window, interface -> medium-2 window."""
    n_p, n_i = int(cfg["piston"]["n"]), int(cfg["interfaces"][0]["n"])
    n_w = int(cfg["grid_water"]["nx"]) * int(cfg["grid_water"]["nz"])
    n_s = int(cfg["grid_solid"]["nx"]) * int(cfg["grid_solid"]["nz"])
    return n_p * n_i + n_p * n_w + n_i * n_w + n_i * n_s


def same_geometry(cfgs) -> bool:
    """True when workloads differ only in frequency (same seed, points, media
    and image grid), so their stages can share every pair's geometry."""
    strip = lambda c: {k: v for k, v in c.items() if k not in ("freq", "name")}
    return len(cfgs) > 1 and all(strip(c) == strip(cfgs[0]) for c in cfgs[1:])


def run_chain_multi(cfgs: list, fmt: str = "c128", workspace: Workspace | None = None,
                    stage_opts: dict | None = None, stream=None, device="cuda") -> list:
    """The chains of 2-4 workloads that differ only in frequency, every stage
    evaluated for all frequencies at once (rsi_propagate_stage_multi).
    Returns one image per workload, as run_chain would."""
    if not same_geometry(cfgs) or not 2 <= len(cfgs) <= 4:
        raise ValueError("run_chain_multi needs 2-4 workloads that differ only in frequency")
    cfg = cfgs[0]
    if cfg.get("precision", "fp32c") != "fp32c":
        raise ValueError("run_chain_multi is FP32C only")
    opts = {k: v for k, v in (stage_opts or {}).items() if k != "variant"}
    ws = workspace or Workspace(device)
    seed = int(cfg.get("seed", 0))
    v0 = float(cfg.get("v0", 1.0))
    media = cfg["media"]
    C = snell_invariant(cfg)
    mode = cfg.get("tmode", "global")
    freqs = [float(c["freq"]) for c in cfgs]
    nf = len(freqs)
    pc = cfg["piston"]
    piston = make_qmc_points(dict({"kind": "disk"}, **pc), seed, int(pc.get("set_id", 0)), int(pc["n"]),
                             device=device, stream=stream)
    ifaces = [make_qmc_points(it, seed, int(it["set_id"]), int(it["n"]), device=device, stream=stream)
              for it in cfg["interfaces"]]
    targets = grid_points(cfg["grid"], device=device, stream=stream)
    first_tgt = ifaces[0] if ifaces else targets
    ks = [wavenumber(f, media[0]["c"]) for f in freqs]
    st = stage_struct(STAGE_PISTON, "fp32c", ks[0], v0, **opts)
    phi = propagate_stage_multi(st, ks, piston, None, first_tgt, workspace=ws, stream=stream)
    for s, pts in enumerate(ifaces):
        sigma = torch.empty_like(phi)
        for f in range(nf):
            interface_transmit(pts, phi[f], media[s], media[s + 1], C, mode, out=sigma[f], stream=stream)
        nxt = ifaces[s + 1] if s + 1 < len(ifaces) else targets
        normals = NORMALS_POINTS if cfg["interfaces"][s]["kind"] != "rect" else NORMALS_Z
        ks = [wavenumber(f, media[s + 1]["c"]) for f in freqs]
        st = stage_struct(STAGE_RSI, "fp32c", ks[0], 1.0, normals, **opts)
        phi = propagate_stage_multi(st, ks, pts, sigma, nxt, workspace=ws, stream=stream)
    k_last = [wavenumber(f, media[len(ifaces)]["c"]) for f in freqs]
    return [field_image(cfg["grid"], phi[f], k_last[f], v0, fmt, stream=stream) for f in range(nf)]


# ---------------------------------------------------------------------------
# batches of single-interface chains in one CUDA graph (rsi_batch_*)
# ---------------------------------------------------------------------------
def batch_instance(cfg: dict) -> BatchInstance:
    """A BatchInstance from a workload description with exactly one interface."""
    if len(cfg["interfaces"]) != 1:
        raise ValueError("batched chains have exactly one interface")
    b = BatchInstance()
    pc, it = cfg["piston"], cfg["interfaces"][0]
    b.piston = surface_struct(dict({"kind": "disk"}, **pc))
    b.iface = surface_struct(it)
    b.n_piston, b.n_iface = int(pc["n"]), int(it["n"])
    b.piston_set, b.iface_set = int(pc.get("set_id", 0)), int(it["set_id"])
    m = cfg["media"]
    b.transmit = interface_struct(m[0], m[1], snell_invariant(cfg), cfg.get("tmode", "global"))
    b.k1 = wavenumber(cfg["freq"], m[0]["c"])
    b.k2 = wavenumber(cfg["freq"], m[1]["c"])
    b.v0 = float(cfg.get("v0", 1.0))
    b.grid = grid_struct(cfg["grid"])
    return b


class Batch:
    """Plan + device buffers of a batch; run() replays one CUDA graph."""

    def __init__(self, cfgs: list, seed: int = 0, shape: Stage | None = None, device="cuda",
                 allocate: bool = True):
        L = load()
        self.cfgs = cfgs
        arr = (BatchInstance * len(cfgs))(*[batch_instance(c) for c in cfgs])
        plan, ws, n_img = ctypes.c_void_p(), ctypes.c_size_t(), ctypes.c_size_t()
        _check(L.rsi_batch_create(arr, len(cfgs), int(seed), ctypes.byref(shape) if shape else None,
                                  ctypes.byref(plan), ctypes.byref(ws), ctypes.byref(n_img)),
               "rsi_batch_create")
        self.plan = plan
        self.workspace_bytes = int(ws.value)
        self.image_elems = int(n_img.value)
        self.offsets = []
        off = 0
        for c in cfgs:
            self.offsets.append(off)
            off += int(c["grid"]["nx"]) * int(c["grid"]["nz"])
        self.ws = self.images = None
        if allocate:
            self.ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=device)
            self.images = torch.empty(self.image_elems, dtype=torch.complex64, device=device)

    def run(self, stream=None) -> torch.Tensor:
        _check(load().rsi_batch_run(self.plan, _ptr(self.ws), self.ws.numel(), _ptr(self.images),
                                    _stream(stream)), "rsi_batch_run")
        return self.images

    def image(self, i: int) -> torch.Tensor:
        g = self.cfgs[i]["grid"]
        n = int(g["nx"]) * int(g["nz"])
        return self.images[self.offsets[i]:self.offsets[i] + n].view(int(g["nz"]), int(g["nx"]))

    def close(self):
        if self.plan:
            load().rsi_batch_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# surrogate building blocks (rsi_nn_*)
# ---------------------------------------------------------------------------
def nn_features(p, lo, hi, fmat, out, stream=None):
    _check(load().rsi_nn_features(_ptr(p), _ptr(lo), _ptr(hi), _ptr(fmat), p.shape[0], p.shape[1],
                                  fmat.shape[0], _ptr(out), _stream(stream)), "rsi_nn_features")
    return out


def nn_gemm(epi: str, A, B, out_f32=None, out_bf16=None, bias=None, aux=None, splits: int = 1,
            workspace=None, engine: str = "mma_sync", a_t: bool = False, b_t: bool = False, stream=None):
    """C[M x N] = A[M x K] B[N x K]^T with an epilogue (see rsi_nn_gemm).
    a_t: A is given as its transpose [K x M]; b_t: B is given as [K x N]."""
    K, M = A.shape if a_t else A.shape[::-1]
    N = B.shape[1] if b_t else B.shape[0]
    assert (B.shape[0] if b_t else B.shape[1]) == K
    if splits > 1:
        assert workspace is not None and workspace.numel() >= splits * M * N
    layout = (1 if a_t else 0) | (2 if b_t else 0)
    _check(load().rsi_nn_gemm(NN_EPI[epi], NN_ENGINE[engine], layout, _ptr(A), _ptr(B), M, N, K, _ptr(bias),
                              _ptr(aux), _ptr(out_f32), _ptr(out_bf16), int(splits), _ptr(workspace),
                              _stream(stream)), "rsi_nn_gemm")


def nn_transpose(x, out, stream=None):
    _check(load().rsi_nn_transpose(_ptr(x), x.shape[0], x.shape[1], _ptr(out), _stream(stream)),
           "rsi_nn_transpose")
    return out


def nn_loss(y, t, grad_scale, grad, partial, loss_out, stream=None):
    _check(load().rsi_nn_loss(_ptr(y), _ptr(t), y.numel(), float(grad_scale), _ptr(grad),
                              _ptr(partial), partial.numel(), _ptr(loss_out), _stream(stream)),
           "rsi_nn_loss")


def nn_colsum(m, out, stream=None):
    _check(load().rsi_nn_colsum(_ptr(m), m.shape[0], m.shape[1], _ptr(out), _stream(stream)),
           "rsi_nn_colsum")


def nn_adam(w, m, v, g, lr, step, w_bf16=None, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().rsi_nn_adam(_ptr(w), _ptr(m), _ptr(v), _ptr(g), w.numel(), float(lr), float(beta1),
                              float(beta2), float(eps), int(step), _ptr(w_bf16), _stream(stream)),
           "rsi_nn_adam")


def nn_adam_dev(w, m, v, g, hyper, w_bf16=None, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """Adam with (lr, 1 - beta1^t, 1 - beta2^t) read from the device tensor
    `hyper` (f32 [3]) when the kernel runs."""
    _check(load().rsi_nn_adam_dev(_ptr(w), _ptr(m), _ptr(v), _ptr(g), w.numel(), _ptr(hyper), float(beta1),
                                  float(beta2), float(eps), _ptr(w_bf16), _stream(stream)), "rsi_nn_adam_dev")


def nn_cast_bf16(x, out, stream=None):
    _check(load().rsi_nn_cast_bf16(_ptr(x), x.numel(), _ptr(out), _stream(stream)), "rsi_nn_cast_bf16")
    return out


def nn_carrier_coeffs(params64, c1: float, c2: float, carrier, params32, stream=None):
    """The surrogate's carrier coefficients (f64 [B, 4]) and its f32 inputs
    from f64 parameter rows [B, 5], on the device."""
    _check(load().rsi_nn_carrier_coeffs(_ptr(params64), params64.shape[0], float(c1), float(c2), _ptr(carrier),
                                        _ptr(params32), _stream(stream)), "rsi_nn_carrier_coeffs")
    return carrier


def nn_gemm_carrier(a, b, bias, carrier, window: dict, sign: int, scale: float, out, workspace=None,
                    stream=None):
    """out = scale * exp(sign i psi) * (a b^T + bias) row by row (tcgen05
    engine): the output layer and the carrier pass in one kernel.  workspace:
    f32 tensor of at least 8 a.shape[0] elements (allocated here if None)."""
    if workspace is None:
        workspace = torch.empty(8 * a.shape[0], dtype=torch.float32, device=a.device)
    G = grid_struct(window)
    _check(load().rsi_nn_gemm_carrier(_ptr(a), _ptr(b), a.shape[0], b.shape[0], a.shape[1], _ptr(bias),
                                      _ptr(carrier), ctypes.byref(G), int(sign), float(scale), _ptr(out),
                                      _ptr(workspace), _stream(stream)), "rsi_nn_gemm_carrier")
    return out


def nn_carrier(carrier, window: dict, sign: int, x, out, stream=None, scale: float = 1.0):
    G = grid_struct(window)
    _check(load().rsi_nn_carrier(_ptr(carrier), carrier.shape[0], ctypes.byref(G), int(sign), float(scale),
                                 _ptr(x), _ptr(out), _stream(stream)), "rsi_nn_carrier")
    return out


# ---------------------------------------------------------------------------
# the surrogate's coordinate network (rsi_nn_rows / forward / backward /
# adam_step / targets / infer)
# ---------------------------------------------------------------------------
NN_ROWS = {"random": 0, "pixels": 1}


def nn_net_struct(n_freq: int, width: int, depth: int, rows: int, engine: str, c1: float, c2: float, a: float,
                  box_lo, box_hi, window: dict, fmat) -> NNNet:
    n = NNNet()
    n.n_freq, n.width, n.depth, n.rows = int(n_freq), int(width), int(depth), int(rows)
    n.engine = NN_ENGINE[engine]
    n.c1, n.c2, n.a = float(c1), float(c2), float(a)
    for k in range(4):
        n.box_lo[k], n.box_hi[k] = float(box_lo[k]), float(box_hi[k])
    n.window = grid_struct(window)
    n.fmat = fmat.data_ptr()
    return n


def nn_param_elems(net: NNNet) -> int:
    v = int(load().rsi_nn_param_elems(ctypes.byref(net)))
    if v < 0:
        raise RSIError("rsi_nn_param_elems", -1, load().rsi_last_error().decode(errors="replace"))
    return v


def nn_param_offset(net: NNNet, layer: int, bias: bool) -> int:
    return int(load().rsi_nn_param_offset(ctypes.byref(net), int(layer), 1 if bias else 0))


def nn_act_bytes(net: NNNet) -> int:
    v = int(load().rsi_nn_act_bytes(ctypes.byref(net)))
    if v == 0:
        raise RSIError("rsi_nn_act_bytes", -1, load().rsi_last_error().decode(errors="replace"))
    return v


def nn_rows(net: NNNet, params64, n_fields: int, mode: str, act, seed: int = 0, seed_dev=None, first: int = 0,
            targets=None, log_rms=None, stream=None):
    _check(load().rsi_nn_rows(ctypes.byref(net), _ptr(params64), int(n_fields), NN_ROWS[mode],
                              int(seed) & (2**64 - 1), _ptr(seed_dev), int(first), _ptr(targets), _ptr(log_rms),
                              _ptr(act), act.numel(), _stream(stream)), "rsi_nn_rows")


def nn_forward(net: NNNet, w16, w32, act, y=None, stream=None):
    _check(load().rsi_nn_forward(ctypes.byref(net), _ptr(w16), _ptr(w32), _ptr(act), act.numel(), _ptr(y),
                                 _stream(stream)), "rsi_nn_forward")


def nn_backward(net: NNNet, w16, w32, act, grad, loss_dev, stream=None):
    _check(load().rsi_nn_backward(ctypes.byref(net), _ptr(w16), _ptr(w32), _ptr(act), act.numel(), _ptr(grad),
                                  _ptr(loss_dev), _stream(stream)), "rsi_nn_backward")


def nn_adam_step(net: NNNet, w32, m, v, grad, w16, hyper, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().rsi_nn_adam_step(ctypes.byref(net), _ptr(w32), _ptr(m), _ptr(v), _ptr(grad), _ptr(w16),
                                   _ptr(hyper), float(beta1), float(beta2), float(eps), _stream(stream)),
           "rsi_nn_adam_step")


def nn_targets(net: NNNet, params64, images, carrier, params32, env, targets, log_rms, stream=None):
    _check(load().rsi_nn_targets(ctypes.byref(net), _ptr(params64), int(params64.shape[0]), _ptr(images),
                                 _ptr(carrier), _ptr(params32), _ptr(env), _ptr(targets), _ptr(log_rms),
                                 _stream(stream)), "rsi_nn_targets")


def nn_infer(net: NNNet, w16, w32, params64, act, carrier, out, stream=None):
    _check(load().rsi_nn_infer(ctypes.byref(net), _ptr(w16), _ptr(w32), _ptr(params64), int(params64.shape[0]),
                               _ptr(act), act.numel(), _ptr(carrier), _ptr(out), _stream(stream)), "rsi_nn_infer")
