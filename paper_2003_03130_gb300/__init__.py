"""GB300 cell/fluid time step: Mooney-Rivlin tet forces, immersed-boundary
coupling and D3Q19 lattice Boltzmann, all in the CUDA library
``libcellfsi.so`` (C ABI in ``include/cellfsi.h``).

This module only marshals arguments to that library through ctypes; every
step of the computation runs in its kernels. There is no CPU fallback: if the
library has not been built, importing the binding fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcellfsi.so")

STATUS = {
    0: "CF_OK", 1: "CF_EINVAL", 2: "CF_EDEGENERATE", 3: "CF_EINVERTED", 4: "CF_ENONFINITE",
    5: "CF_EDOMAIN", 6: "CF_ESTATE", 7: "CF_ECUDA", 8: "CF_ETIMEOUT", 9: "CF_ENOMEM", 10: "CF_EUNSTABLE",
}


class CellFSIError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.name = STATUS.get(status, str(status))


_lib = None
_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int32)


def lib():
    """The loaded CUDA library (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        vp = ctypes.c_void_p
        sig = {
            "cf_create": ([ctypes.POINTER(vp), ctypes.c_int, vp], ctypes.c_int),
            "cf_destroy": ([vp], None),
            "cf_set_population_format": ([vp, ctypes.c_int32], ctypes.c_int),
            "cf_set_delta": ([vp, ctypes.c_int32], ctypes.c_int),
            "cf_set_spread": ([vp, ctypes.c_int32], ctypes.c_int),
            "cf_lbm_init": ([vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                             ctypes.c_double, _d], ctypes.c_int),
            "cf_mesh_init": ([vp, ctypes.c_int32, _d, ctypes.c_int32, _i, _d, _i], ctypes.c_int),
            "cf_mesh_init_batch": ([vp, ctypes.c_int32, _i, _d, _i, _i, _d, _i], ctypes.c_int),
            "cf_set_materials": ([vp, ctypes.c_int32, _i, _d, _d, _d], ctypes.c_int),
            "cf_set_tet_materials": ([vp, ctypes.c_int32, _i, ctypes.c_int32, _d, _d, _d], ctypes.c_int),
            "cf_set_material": ([vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double], ctypes.c_int),
            "cf_step": ([vp, ctypes.c_int32], ctypes.c_int),
            "cf_step_async": ([vp, ctypes.c_int32], ctypes.c_int),
            "cf_prepare_steps": ([vp, ctypes.c_int32], ctypes.c_int),
            "cf_step_exchange": ([vp, ctypes.c_int32, vp, vp], ctypes.c_int),  # addresses: the per-step call
            "cf_get_launch_shape": ([vp, _i], ctypes.c_int),
            "cf_set_launch_shape": ([vp, _i], ctypes.c_int),
            "cf_autotune": ([vp, ctypes.c_int32, _i], ctypes.c_int),
            "cf_set_chain_wait": ([vp, ctypes.c_int64, ctypes.c_int32], ctypes.c_int),
            "cf_synchronize": ([vp], ctypes.c_int),
            "cf_compute_forces": ([vp], ctypes.c_int),
            "cf_step_profiled": ([vp, ctypes.c_int32, _d, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
            "cf_get_forces": ([vp, ctypes.c_int32, _d], ctypes.c_int),
            "cf_get_positions": ([vp, ctypes.c_int32, _d], ctypes.c_int),
            "cf_set_positions": ([vp, ctypes.c_int32, _d], ctypes.c_int),
            "cf_get_velocity": ([vp, _d], ctypes.c_int),
            "cf_get_density": ([vp, _d], ctypes.c_int),
            "cf_get_energy": ([vp, ctypes.c_int32, _d], ctypes.c_int),
            "cf_get_csr": ([vp, ctypes.c_int32, _i, _i], ctypes.c_int),
            "cf_get_taylor": ([vp, ctypes.c_int32, _d], ctypes.c_int),
            "cf_get_cell_strain": ([vp, ctypes.c_int32, ctypes.c_double, _d], ctypes.c_int),
            "cf_get_mesh": ([vp, ctypes.c_int32, _i, _d, _d], ctypes.c_int),
            "cf_cell_verts": ([vp, ctypes.c_int32], ctypes.c_int32),
            "cf_cell_tets": ([vp, ctypes.c_int32], ctypes.c_int32),
            "cf_last_error": ([vp], ctypes.c_char_p),
            "cf_plates_set": ([vp, ctypes.c_double, _d, _d], ctypes.c_int),
            "cf_relax": ([vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_int32], ctypes.c_int),
            "cf_plate_force": ([vp, _d], ctypes.c_int),
            "cf_tape_clear": ([vp], ctypes.c_int),
            "cf_tape_generation": ([vp, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
            "cf_relax_adjoint": ([vp, _d], ctypes.c_int),
            "cf_adjoint_gradients": ([vp, _d], ctypes.c_int),
            "cf_force_jvp": ([vp, _d, _d], ctypes.c_int),
            "cf_force_param_vjp": ([vp, _d, _d], ctypes.c_int),
            "cf_vertex_forces_static": ([ctypes.c_int32, ctypes.c_int32, vp, vp, vp, vp, vp, vp, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, vp, vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(ctx, status: int):
    if status != 0:
        msg = lib().cf_last_error(ctx.handle if ctx is not None else None)
        raise CellFSIError(status, (msg or b"").decode())


def _p(a, t=_d):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _out(out, shape, dtype=np.float64):
    if out is None:
        return np.empty(shape, dtype)
    if out.shape != tuple(shape) or out.dtype != dtype or not out.flags.c_contiguous:
        raise ValueError(f"output must be a C-contiguous {dtype} array of shape {shape}")
    return out


class Context:
    """Holds a ``cf_ctx*`` and the sizes needed to shape outputs."""

    def __init__(self, handle, device):
        self.handle = handle
        self.device = device
        self.dims = None  # (nx, ny, nz)

    def __del__(self):
        try:
            cf_destroy(self)
        except Exception:
            pass


def _default_stream(device: int):
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream(device).cuda_stream or None
    except ImportError:
        pass
    return None


def cf_create(device: int = 0, stream=None) -> Context:
    """``stream``: a cudaStream_t handle (int); default PyTorch's current
    stream on ``device`` (the library makes its own if that is the legacy
    default stream)."""
    h = ctypes.c_void_p()
    s = _default_stream(device) if stream is None else (stream or None)
    st = lib().cf_create(ctypes.byref(h), device, s)
    if st != 0:
        raise CellFSIError(st, "cf_create failed")
    return Context(h, device)


def cf_destroy(ctx: Context):
    if ctx.handle:
        lib().cf_destroy(ctx.handle)
        ctx.handle = None


def cf_last_error(ctx) -> str:
    return (lib().cf_last_error(ctx.handle) or b"").decode()


CF_POP_F32, CF_POP_F16, CF_POP_BF16, CF_POP_F16_SR, CF_POP_BF16_SR = 0, 1, 2, 3, 4
CF_ALL_CELLS = -1
POP_FORMATS = {"f32": CF_POP_F32, "f16": CF_POP_F16, "bf16": CF_POP_BF16, "f16sr": CF_POP_F16_SR,
               "bf16sr": CF_POP_BF16_SR}


def cf_set_population_format(ctx, fmt):
    """``fmt``: a CF_POP_* code or "f32" / "f16" / "bf16" / "f16sr" /
    "bf16sr" (the last two round stochastically); applies at the next
    cf_lbm_init."""
    fmt = POP_FORMATS.get(fmt, fmt)
    _check(ctx, lib().cf_set_population_format(ctx.handle, int(fmt)))


CF_DELTA_TRILINEAR, CF_DELTA_PESKIN4 = 2, 4
DELTAS = {"trilinear": CF_DELTA_TRILINEAR, "peskin4": CF_DELTA_PESKIN4}


def cf_set_delta(ctx, kernel):
    """``kernel``: CF_DELTA_TRILINEAR / CF_DELTA_PESKIN4 (the support width,
    2 or 4) or "trilinear" / "peskin4"; applies at the next cf_lbm_init."""
    kernel = DELTAS.get(kernel, kernel)
    _check(ctx, lib().cf_set_delta(ctx.handle, int(kernel)))


CF_SPREAD_FLOAT, CF_SPREAD_FIXED = 0, 1
SPREADS = {"float": CF_SPREAD_FLOAT, "fixed": CF_SPREAD_FIXED}


def cf_set_spread(ctx, mode):
    """``mode``: CF_SPREAD_FLOAT / CF_SPREAD_FIXED or "float" / "fixed" (the
    deterministic fixed-point force field); applies at the next cf_lbm_init."""
    mode = SPREADS.get(mode, mode)
    _check(ctx, lib().cf_set_spread(ctx.handle, int(mode)))


def cf_lbm_init(ctx, nx, ny, nz, tau, u_wall_lo_x, u_wall_hi_x, body_force=None):
    g = None if body_force is None else _f64(body_force).reshape(3)
    _check(ctx, lib().cf_lbm_init(ctx.handle, nx, ny, nz, tau, u_wall_lo_x, u_wall_hi_x, _p(g)))
    ctx.dims = (nx, ny, nz)


def cf_mesh_init(ctx, x_ref, tets, y0=None) -> int:
    x = _f64(x_ref).reshape(-1, 3)
    t = np.ascontiguousarray(tets, dtype=np.int32).reshape(-1, 4)
    y = None if y0 is None else _f64(y0).reshape(-1, 3)
    if y is not None and y.shape != x.shape:
        raise ValueError("y0 must have the shape of x_ref")
    cid = ctypes.c_int32(-1)
    _check(ctx, lib().cf_mesh_init(ctx.handle, len(x), _p(x), len(t), _p(t, _i), _p(y), ctypes.byref(cid)))
    return cid.value


def cf_mesh_init_batch(ctx, cells_x_ref, cells_tets, cells_y0=None):
    """Add several cells at once: lists of per-cell ``x_ref [nv,3]``,
    ``tets [nt,4]`` (local indices) and optionally ``y0``. Returns the ids."""
    xs = [_f64(x).reshape(-1, 3) for x in cells_x_ref]
    ts = [np.ascontiguousarray(t, dtype=np.int32).reshape(-1, 4) for t in cells_tets]
    nv = np.array([len(x) for x in xs], np.int32)
    nt = np.array([len(t) for t in ts], np.int32)
    x = np.ascontiguousarray(np.concatenate(xs))
    t = np.ascontiguousarray(np.concatenate(ts))
    y = None if cells_y0 is None else np.ascontiguousarray(np.concatenate([_f64(v).reshape(-1, 3) for v in cells_y0]))
    ids = np.zeros(len(xs), np.int32)
    _check(ctx, lib().cf_mesh_init_batch(ctx.handle, len(xs), _p(nv, _i), _p(x), _p(nt, _i), _p(t, _i), _p(y),
                                         _p(ids, _i)))
    return ids.tolist()


def cf_set_materials(ctx, ids, mu, kappa, w):
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    mu, kappa, w = _f64(mu), _f64(kappa), _f64(w)
    _check(ctx, lib().cf_set_materials(ctx.handle, len(ids), _p(ids, _i), _p(mu), _p(kappa), _p(w)))


def cf_set_material(ctx, cell_id, mu, kappa, w):
    _check(ctx, lib().cf_set_material(ctx.handle, cell_id, mu, kappa, w))


def cf_set_tet_materials(ctx, cell_id, region, mu, kappa, w):
    """Per-tet materials of one cell: ``region`` [nt] in [0, nreg), and
    ``mu``, ``kappa``, ``w`` [nreg]."""
    region = np.ascontiguousarray(region, dtype=np.int32).reshape(-1)
    mu, kappa, w = _f64(np.atleast_1d(mu)), _f64(np.atleast_1d(kappa)), _f64(np.atleast_1d(w))
    if not (len(mu) == len(kappa) == len(w)):
        raise ValueError("mu, kappa, w need one value per region")
    nt = lib().cf_cell_tets(ctx.handle, cell_id)
    if nt > 0 and len(region) != nt:
        raise ValueError(f"region needs one entry per tet of the cell ({nt})")
    _check(ctx, lib().cf_set_tet_materials(ctx.handle, cell_id, _p(region, _i), len(mu), _p(mu), _p(kappa), _p(w)))


def cf_step(ctx, n: int = 1):
    _check(ctx, lib().cf_step(ctx.handle, n))


def cf_step_async(ctx, n: int = 1):
    _check(ctx, lib().cf_step_async(ctx.handle, n))


def cf_step_exchange(ctx, n: int, y_in=None, out=None):
    """Set all positions from ``y_in`` [V,3] (or keep them when None),
    advance n steps, and return all positions (into ``out`` when given),
    with one wait."""
    L = lib()
    nv = L.cf_cell_verts(ctx.handle, CF_ALL_CELLS)
    pi = None
    if y_in is not None:
        yi = _f64(y_in)
        if yi.size != 3 * nv:
            raise ValueError(f"y_in must hold {nv} x 3 positions")
        pi = yi.ctypes.data
    yo = _out(out, (nv, 3))
    _check(ctx, L.cf_step_exchange(ctx.handle, n, pi, yo.ctypes.data))
    return yo


def cf_prepare_steps(ctx, n: int):
    """Instantiate the step graphs an n-step call would use, without running."""
    _check(ctx, lib().cf_prepare_steps(ctx.handle, n))


CF_SHAPE_LEN = 15
SHAPE_KEYS = ("tile_x", "tile_y", "tile_z", "tet_block", "gather_block", "interp_block", "fused", "near_rows",
              "far_spec", "tet_form", "pop_l2", "pop_pairs", "mark_k5", "staged", "interp_form")


def cf_get_launch_shape(ctx):
    """The launch shape as a dict over SHAPE_KEYS."""
    out = np.zeros(CF_SHAPE_LEN, np.int32)
    _check(ctx, lib().cf_get_launch_shape(ctx.handle, _p(out, _i)))
    return dict(zip(SHAPE_KEYS, (int(v) for v in out)))


def cf_set_launch_shape(ctx, shape):
    """``shape``: a dict over SHAPE_KEYS (missing keys keep their value) or
    CF_SHAPE_LEN ints; applies from the next step call."""
    if isinstance(shape, dict):
        cur = cf_get_launch_shape(ctx)
        cur.update(shape)
        shape = [cur[k] for k in SHAPE_KEYS]
    arr = np.ascontiguousarray(shape, np.int32)
    if arr.shape != (CF_SHAPE_LEN,):
        raise ValueError(f"need {CF_SHAPE_LEN} values")
    _check(ctx, lib().cf_set_launch_shape(ctx.handle, _p(arr, _i)))


def cf_autotune(ctx, steps_per_candidate=20):
    """Time the launch-shape candidates on the context's own state, each as
    steps_per_candidate whole coupled steps run like cf_step (the
    simulation advances 32 x steps_per_candidate steps), and keep the
    fastest; returns the chosen shape."""
    out = np.zeros(CF_SHAPE_LEN, np.int32)
    _check(ctx, lib().cf_autotune(ctx.handle, steps_per_candidate, _p(out, _i)))
    return dict(zip(SHAPE_KEYS, (int(v) for v in out)))


def cf_set_chain_wait(ctx, max_polls=1 << 24, extra_need=0):
    """Bounds of the fused cell chain's waits; extra_need > 0 makes every
    wait unreachable (tests of the CF_ETIMEOUT path)."""
    _check(ctx, lib().cf_set_chain_wait(ctx.handle, int(max_polls), int(extra_need)))


def cf_synchronize(ctx):
    _check(ctx, lib().cf_synchronize(ctx.handle))


def cf_step_profiled(ctx, n: int):
    """Mean ms per step of [tet force, gather + spread, far-field LBM,
    near-field LBM, interpolate + advect] over n directly launched steps,
    and the number of nodes in the force region."""
    ms = np.zeros(5)
    near = ctypes.c_int64(0)
    _check(ctx, lib().cf_step_profiled(ctx.handle, n, _p(ms), ctypes.byref(near)))
    return ms, near.value


def cf_compute_forces(ctx):
    _check(ctx, lib().cf_compute_forces(ctx.handle))


def cf_cell_verts(ctx, cell_id) -> int:
    return lib().cf_cell_verts(ctx.handle, cell_id)


def cf_cell_tets(ctx, cell_id) -> int:
    return lib().cf_cell_tets(ctx.handle, cell_id)


def cf_get_forces(ctx, cell_id, out=None):
    o = _out(out, (cf_cell_verts(ctx, cell_id), 3))
    _check(ctx, lib().cf_get_forces(ctx.handle, cell_id, _p(o)))
    return o


def cf_get_positions(ctx, cell_id, out=None):
    o = _out(out, (cf_cell_verts(ctx, cell_id), 3))
    _check(ctx, lib().cf_get_positions(ctx.handle, cell_id, _p(o)))
    return o


def cf_set_positions(ctx, cell_id, y):
    y = _f64(y)
    if y.shape != (cf_cell_verts(ctx, cell_id), 3):
        raise ValueError("positions must be [nv, 3]")
    _check(ctx, lib().cf_set_positions(ctx.handle, cell_id, _p(y)))


def cf_get_velocity(ctx, out=None):
    nx, ny, nz = ctx.dims
    o = _out(out, (nz, ny, nx, 3))
    _check(ctx, lib().cf_get_velocity(ctx.handle, _p(o)))
    return o


def cf_get_density(ctx, out=None):
    nx, ny, nz = ctx.dims
    o = _out(out, (nz, ny, nx))
    _check(ctx, lib().cf_get_density(ctx.handle, _p(o)))
    return o


def cf_get_energy(ctx, cell_id) -> float:
    e = ctypes.c_double()
    _check(ctx, lib().cf_get_energy(ctx.handle, cell_id, ctypes.byref(e)))
    return e.value


TAYLOR_KEYS = ("D", "D_literal", "inclination", "a1", "a2", "a3", "theta1", "theta2", "theta3", "volume")


def cf_get_taylor(ctx, cell_id):
    """Taylor deformation of a cell (computed on the device), as a dict."""
    out = np.zeros(10)
    _check(ctx, lib().cf_get_taylor(ctx.handle, cell_id, _p(out)))
    return dict(zip(TAYLOR_KEYS, out.tolist()))


def cf_get_cell_strain(ctx, cell_id, d_ref):
    """Cell strain (computed on the device): {"d_max": largest vertex-vertex
    distance, "strain": (d_max - d_ref) / d_ref}."""
    out = np.zeros(2)
    _check(ctx, lib().cf_get_cell_strain(ctx.handle, cell_id, float(d_ref), _p(out)))
    return {"d_max": float(out[0]), "strain": float(out[1])}


def cf_get_csr(ctx, cell_id):
    nv, nt = cf_cell_verts(ctx, cell_id), cf_cell_tets(ctx, cell_id)
    ptr = np.empty(nv + 1, np.int32)
    idx = np.empty(4 * nt, np.int32)
    _check(ctx, lib().cf_get_csr(ctx.handle, cell_id, _p(ptr, _i), _p(idx, _i)))
    return ptr, idx


def cf_get_mesh(ctx, cell_id):
    nt = cf_cell_tets(ctx, cell_id)
    tets = np.empty((nt, 4), np.int32)
    B = np.empty((nt, 3, 3))
    V0 = np.empty(nt)
    _check(ctx, lib().cf_get_mesh(ctx.handle, cell_id, _p(tets, _i), _p(B), _p(V0)))
    return tets, B, V0


def cf_vertex_forces_static(nv, nt, tets, B, V0, u, csr_ptr, csr_idx, mu, kappa, w, f, stream=None):
    """Vertex forces of one cell without a context and without any device
    allocation. Every array argument is a DEVICE address (int) in the
    layouts of ``cf_vertex_forces_static`` in include/cellfsi.h; ``stream``
    is a cudaStream_t handle (int) or None."""
    st = lib().cf_vertex_forces_static(nv, nt, tets, B, V0, u, csr_ptr, csr_idx, mu, kappa, w, f, stream or None)
    if st != 0:
        raise CellFSIError(st, "cf_vertex_forces_static failed")


def _ncells(ctx):
    n = 0
    while cf_cell_verts(ctx, n) > 0:
        n += 1
    return n


def cf_plates_set(ctx, k_plate, z_lo, z_hi):
    zlo, zhi = _f64(z_lo).reshape(-1), _f64(z_hi).reshape(-1)
    _check(ctx, lib().cf_plates_set(ctx.handle, k_plate, _p(zlo), _p(zhi)))


def cf_relax(ctx, n, dt, damping=0.0, record=False):
    _check(ctx, lib().cf_relax(ctx.handle, n, dt, damping, 1 if record else 0))


def cf_plate_force(ctx):
    out = np.zeros(_ncells(ctx))
    _check(ctx, lib().cf_plate_force(ctx.handle, _p(out)))
    return out


def cf_tape_clear(ctx):
    _check(ctx, lib().cf_tape_clear(ctx.handle))


def cf_tape_generation(ctx):
    out = ctypes.c_int64(0)
    _check(ctx, lib().cf_tape_generation(ctx.handle, ctypes.byref(out)))
    return int(out.value)


def cf_relax_adjoint(ctx, dF):
    dF = _f64(dF).reshape(-1)
    _check(ctx, lib().cf_relax_adjoint(ctx.handle, _p(dF)))


def cf_adjoint_gradients(ctx):
    out = np.zeros((_ncells(ctx), 3))
    _check(ctx, lib().cf_adjoint_gradients(ctx.handle, _p(out)))
    return out


def cf_force_jvp(ctx, v):
    v = _f64(v).reshape(-1, 3)
    out = np.zeros_like(v)
    _check(ctx, lib().cf_force_jvp(ctx.handle, _p(v), _p(out)))
    return out


def cf_force_param_vjp(ctx, lam):
    lam = _f64(lam).reshape(-1, 3)
    out = np.zeros((_ncells(ctx), 3))
    _check(ctx, lib().cf_force_param_vjp(ctx.handle, _p(lam), _p(out)))
    return out


def load_workload(ctx, wl):
    """Set up a :class:`workloads.configs.Workload` on the device: fluid, then
    every cell with its material. Returns the cell ids."""
    cf_set_delta(ctx, getattr(wl, "delta", CF_DELTA_TRILINEAR))
    cf_lbm_init(ctx, wl.nx, wl.ny, wl.nz, wl.tau, wl.u_wall_lo, wl.u_wall_hi, wl.body_force)
    if not wl.cells:
        return []
    ids = cf_mesh_init_batch(ctx, [c.x_ref for c in wl.cells], [c.tets for c in wl.cells], [c.y0 for c in wl.cells])
    cf_set_materials(ctx, ids, [c.mu for c in wl.cells], [c.kappa for c in wl.cells], [c.w for c in wl.cells])
    for i, c in zip(ids, wl.cells):
        if getattr(c, "regions", None) is not None:
            m = np.asarray(c.region_materials, np.float64).reshape(-1, 3)
            cf_set_tet_materials(ctx, i, c.regions, m[:, 0], m[:, 1], m[:, 2])
    return ids
