"""Plain FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(its ``cpu_baseline`` and ``--impl reference``) may import this package. It shares no code with the CUDA path:
the arithmetic lives in ``oracle.c`` (compiled with gcc into
``liboracle.so``) and in the plain numpy diagnostics of ``analysis.py``.

The coupled time step here strings the C routines together in the order
t -> t+1 (Sec. 6 gives no explicit order; this is the reading used
throughout):

1. elastic forces from the current positions y^t (Sec. 3.1);
2. spread the vertex forces onto the lattice, F(t);
3. one lattice-Boltzmann step with F(t), which also yields u(t);
4. interpolate u(t) at y^t;
5. y^{t+1} = y^t + u (massless vertices, explicit Euler, dt = 1).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (plain -O2, single thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.ora_mr_eval.argtypes = [_d, ctypes.c_double, ctypes.c_double, ctypes.c_double, _d, _d, _d, _d, _d]
        L.ora_mesh_prepare.argtypes = [ctypes.c_int32, _d, ctypes.c_int32, _i, _d, _d, _i]
        L.ora_mesh_prepare.restype = ctypes.c_int
        L.ora_csr.argtypes = [ctypes.c_int32, ctypes.c_int32, _i, _i, _i]
        L.ora_tet_force.argtypes = [ctypes.c_int32, ctypes.c_int32, _i, _d, _d, _d, _i, _d, _d, _d, _d, _d]
        L.ora_gather.argtypes = [ctypes.c_int32, ctypes.c_int32, _i, _i, _d, _d]
        L.ora_spread.argtypes = [ctypes.c_int32, ctypes.c_int32, _d, _d, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, _d]
        L.ora_spread.restype = ctypes.c_int
        L.ora_interp.argtypes = [ctypes.c_int32, ctypes.c_int32, _d, _d, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, _d]
        L.ora_interp.restype = ctypes.c_int
        L.ora_lbm_velocities.argtypes = [_i, _d]
        L.ora_lbm_equilibrium.argtypes = [ctypes.c_int64, ctypes.c_double, _d, _d]
        L.ora_lbm_step.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, _d, _d, _d, _d, _d, _d, ctypes.c_int64, ctypes.c_int64]
        _lib = L
    return _lib


def _p(a, t=_d):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------- mechanics

TABLE_NAMES = ("J", "T_C", "T_C2", "I", "K", "U", "dU_dI", "dI_dTC", "dU_dK", "dK_dTC",
               "dI_dJ", "dK_dJ", "dU_dJ", "dK_dTC2")


def mr_eval(F, mu1, mu2, kappa):
    """Invariants, energy density, each derivative-table entry and P = dU/dF
    for one 3x3 deformation gradient (Sec. 2, Sec. 3.2)."""
    F = _f64(F).reshape(9)
    out = np.zeros(14)
    dTC, dJ, dTC2, P = (np.zeros(9) for _ in range(4))
    lib().ora_mr_eval(_p(F), mu1, mu2, kappa, _p(out), _p(dTC), _p(dJ), _p(dTC2), _p(P))
    d = dict(zip(TABLE_NAMES, out.tolist()))
    d.update(dTC_dF=dTC.reshape(3, 3), dJ_dF=dJ.reshape(3, 3), dTC2_dF=dTC2.reshape(3, 3), P=P.reshape(3, 3))
    return d


class MeshError(ValueError):
    def __init__(self, code, tet):
        super().__init__(f"mesh error {code} at tet {tet}")
        self.code, self.tet = code, tet


def mesh_prepare(x, tets):
    """Orient tets, B = J^-1 and V_0 per tet (Sec. 3.2). Returns
    ``(tets_oriented [T,4] int32, B [T,3,3], V0 [T])``."""
    x = _f64(x)
    t = _i32(tets).copy()
    B = np.zeros((len(t), 3, 3))
    V0 = np.zeros(len(t))
    bad = np.zeros(1, np.int32)
    rc = lib().ora_mesh_prepare(len(x), _p(x), len(t), _p(t, _i), _p(B), _p(V0), _p(bad, _i))
    if rc:
        raise MeshError(rc, int(bad[0]))
    return t, B, V0


def csr(nv, tets):
    t = _i32(tets)
    ptr = np.zeros(nv + 1, np.int32)
    idx = np.zeros(4 * len(t), np.int32)
    lib().ora_csr(nv, len(t), _p(t, _i), _p(ptr, _i), _p(idx, _i))
    return ptr, idx


def tet_forces(tets, B, V0, u, cell, mu, kappa, w, energy=False):
    """Corner forces [T,4,3] (and V_0 U per tet) for displacements u [V,3]."""
    tets, B, V0, u = _i32(tets), _f64(B), _f64(V0), _f64(u)
    cell = _i32(cell)
    mu, kappa, w = _f64(np.atleast_1d(mu)), _f64(np.atleast_1d(kappa)), _f64(np.atleast_1d(w))
    fc = np.zeros((len(tets), 4, 3))
    en = np.zeros(len(tets)) if energy else None
    lib().ora_tet_force(0, len(tets), _p(tets, _i), _p(B), _p(V0), _p(u), _p(cell, _i), _p(mu), _p(kappa),
                        _p(w), _p(fc), _p(en))
    return (fc, en) if energy else fc


def gather(ptr, idx, fc):
    ptr, idx, fc = _i32(ptr), _i32(idx), _f64(fc)
    nv = len(ptr) - 1
    f = np.zeros((nv, 3))
    lib().ora_gather(0, nv, _p(ptr, _i), _p(idx, _i), _p(fc), _p(f))
    return f


class Mesh:
    """All cells of a run as one mesh: concatenated vertices and tets,
    per-tet cell index, and a material table (mu, kappa, w): slot c is cell
    c's material; a cell with per-tet regions (Sec. 3.1: the force is local,
    so regions may differ) gets further slots, one per region, and its tets
    point at them through ``tmat``."""

    def __init__(self, cells):
        xs, ts, cid, off = [], [], [], 0
        for c_i, c in enumerate(cells):
            xs.append(_f64(c.x_ref))
            ts.append(_i32(c.tets) + off)
            cid.append(np.full(len(c.tets), c_i, np.int32))
            off += len(c.x_ref)
        self.x = np.concatenate(xs) if xs else np.zeros((0, 3))
        tets = np.concatenate(ts) if ts else np.zeros((0, 4), np.int32)
        self.cell = np.concatenate(cid) if cid else np.zeros(0, np.int32)
        self.tets, self.B, self.V0 = mesh_prepare(self.x, tets)
        self.ptr, self.idx = csr(len(self.x), self.tets)
        mats = [(c.mu, c.kappa, c.w) for c in cells]
        self.tmat = self.cell.copy()
        t0 = 0
        for c in cells:
            if getattr(c, "regions", None) is not None:
                self.tmat[t0:t0 + len(c.tets)] = len(mats) + _i32(c.regions)
                mats += [tuple(m) for m in c.region_materials]
            t0 += len(c.tets)
        self.mu = np.array([m[0] for m in mats], np.float64)
        self.kappa = np.array([m[1] for m in mats], np.float64)
        self.w = np.array([m[2] for m in mats], np.float64)
        self.vert_ranges = []
        o = 0
        for c in cells:
            self.vert_ranges.append((o, o + len(c.x_ref)))
            o += len(c.x_ref)

    def forces(self, y, energy=False):
        """Vertex forces [V,3] at positions y (u = y - x)."""
        r = tet_forces(self.tets, self.B, self.V0, _f64(y) - self.x, self.tmat, self.mu, self.kappa, self.w,
                       energy=energy)
        if energy:
            fc, en = r
            return gather(self.ptr, self.idx, fc), en
        return gather(self.ptr, self.idx, r)

    def energy(self, y):
        _, en = tet_forces(self.tets, self.B, self.V0, _f64(y) - self.x, self.tmat, self.mu, self.kappa,
                           self.w, energy=True)
        return float(en.sum())


# ---------------------------------------------------------------- IBM

class DomainError(ValueError):
    pass


def _width(width):
    if width not in (2, 4):
        raise ValueError("delta support width must be 2 (trilinear) or 4 (Peskin four-point)")
    return width


def spread(y, f, nx, ny, nz, out=None, width=2):
    """F(x) += sum_v f_v delta_h(x - y_v), delta of support width 2 or 4."""
    y, f = _f64(y), _f64(f)
    Fn = np.zeros((nz, ny, nx, 3)) if out is None else out
    bad = lib().ora_spread(0, len(y), _p(y), _p(f), nx, ny, nz, _width(width), _p(Fn))
    if bad:
        raise DomainError(f"{bad} vertices have delta support outside the walls")
    return Fn


def interp(y, ufield, width=2):
    """v(y_v) = sum_x u(x) delta_h(x - y_v), delta of support width 2 or 4."""
    y = _f64(y)
    ufield = _f64(ufield)
    nz, ny, nx, _ = ufield.shape
    v = np.zeros((len(y), 3))
    bad = lib().ora_interp(0, len(y), _p(y), _p(ufield), nx, ny, nz, _width(width), _p(v))
    if bad:
        raise DomainError(f"{bad} vertices have delta support outside the walls")
    return v


# ---------------------------------------------------------------- LBM

def lattice():
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    lib().ora_lbm_velocities(_p(c, _i), _p(w))
    return c, w


class Fluid:
    """D3Q19 BGK fluid with Guo forcing and moving walls (post-collision
    populations ``f [nz,ny,nx,19]``)."""

    def __init__(self, nx, ny, nz, tau, u_wall_lo, u_wall_hi, body_force=(0.0, 0.0, 0.0)):
        self.nx, self.ny, self.nz, self.tau = nx, ny, nz, float(tau)
        self.uw = (float(u_wall_lo), float(u_wall_hi))
        self.g = _f64(body_force)
        self.f = np.zeros((nz, ny, nx, 19))
        u0 = np.zeros(3)
        lib().ora_lbm_equilibrium(nx * ny * nz, 1.0, _p(u0), _p(self.f))
        self.rho = np.ones((nz, ny, nx))
        self.u = np.zeros((nz, ny, nx, 3))

    def step(self, Fn=None, n0=0, n1=None):
        n1 = self.nx * self.ny * self.nz if n1 is None else n1
        fout = np.empty_like(self.f)
        if Fn is not None:
            Fn = _f64(Fn)
        lib().ora_lbm_step(self.nx, self.ny, self.nz, self.tau, self.uw[0], self.uw[1], _p(self.g), _p(self.f),
                           _p(Fn), _p(fout), _p(self.rho), _p(self.u), n0, n1)
        self.f = fout

    def total_mass(self):
        return float(self.f.sum())

    def total_momentum(self):
        c, _ = lattice()
        return np.einsum("zyxi,ia->a", self.f, c.astype(np.float64))


# ---------------------------------------------------------------- coupled

class Coupled:
    """Cells immersed in the fluid; one call of :meth:`step` is t -> t+1."""

    def __init__(self, wl):
        self.fluid = Fluid(wl.nx, wl.ny, wl.nz, wl.tau, wl.u_wall_lo, wl.u_wall_hi, wl.body_force)
        self.mesh = Mesh(wl.cells) if wl.cells else None
        self.y = np.concatenate([_f64(c.y0) for c in wl.cells]) if wl.cells else np.zeros((0, 3))
        self.Fn = np.zeros((wl.nz, wl.ny, wl.nx, 3))
        self.last_forces = np.zeros_like(self.y)
        self.width = getattr(wl, "delta", 2)

    def step(self, n=1):
        fl = self.fluid
        for _ in range(n):
            self.Fn[...] = 0.0
            if self.mesh is not None:
                fv = self.mesh.forces(self.y)                       # 1. elastic forces at y^t
                self.last_forces = fv
                spread(self.y, fv, fl.nx, fl.ny, fl.nz, out=self.Fn, width=self.width)  # 2. F(t)
            fl.step(self.Fn)                                         # 3. LB step, u(t)
            if self.mesh is not None:
                v = interp(self.y, fl.u, width=self.width)          # 4. u(t) at y^t
                self.y = self.y + v                                  # 5. y^{t+1}
