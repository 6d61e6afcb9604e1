"""ctypes front end of the FP64 CPU oracle (``aenet_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's
CPU-baseline leg load this module; the GPU product path never does. The oracle
is plain C compiled with gcc (no CUDA), shares no code with the GPU library and
evaluates the potential exactly as the paper defines it (Sec. II.A, II.B).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aenet_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

BRUTE, CELLS = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no -march flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Model(C.Structure):
    _fields_ = [("n_species", C.c_int), ("type_weight", C.POINTER(C.c_double)),
                ("rc_rad", C.c_double), ("order_rad", C.c_int),
                ("rc_ang", C.c_double), ("order_ang", C.c_int),
                ("n_layers", C.c_int), ("widths", C.POINTER(C.c_int)),
                ("params", C.POINTER(C.c_double)),
                ("in_shift", C.POINTER(C.c_double)), ("in_scale", C.POINTER(C.c_double))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        _lib.orc_compute.argtypes = [C.POINTER(_Model), C.c_int, P, P, P, C.c_int, C.c_int, P,
                                     P, P, P, P, P, P, P]
        _lib.orc_forces_subset.argtypes = [C.POINTER(_Model), C.c_int, P, P, P, C.c_int, C.c_int,
                                           C.c_int, P, P, P]
        _lib.orc_md_nve.argtypes = [C.POINTER(_Model), C.c_int, P, P, P, P, P, C.c_double,
                                    C.c_int, C.c_int, C.c_int, P, P]
        _lib.orc_md_nvt.argtypes = [C.POINTER(_Model), C.c_int, P, P, P, P, P, C.c_double,
                                    C.c_int, C.c_int, C.c_int, P, P, C.c_double, C.c_double]
        _lib.orc_compute_tri.argtypes = [C.POINTER(_Model), C.c_int, P, P, P, P, C.c_int, C.c_int,
                                         P, P, P, P, P]
        _lib.orc_md_tri.argtypes = [C.POINTER(_Model), C.c_int, P, P, P, P, P, P, C.c_double, C.c_int,
                                    C.c_int, P, P, C.c_double, C.c_double]
        _lib.orc_md_npt.argtypes = [C.POINTER(_Model), C.c_int, P, P, P, P, P, P, C.c_double, C.c_int,
                                    C.c_int, P, P, C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_int]
        _lib.orc_neighbour_lists.argtypes = [C.c_int, C.c_int, P, P, C.c_double, P, P, P, P]
        _lib.orc_chebyshev.argtypes = [C.c_int, C.c_double, P, P]
        _lib.orc_chebyshev.restype = None
        _lib.orc_cutoff.argtypes = [C.c_double, C.c_double, P]
        _lib.orc_cutoff.restype = None
    return _lib


def chebyshev(n, x):
    """(T_0..T_n(x), dT_0/dx..dT_n/dx) from the oracle's recurrences."""
    T = np.zeros(n + 1)
    dT = np.zeros(n + 1)
    lib().orc_chebyshev(int(n), float(x), _ptr(T), _ptr(dT))
    return T, dT


def cutoff(r, rc):
    """(f_c(r), df_c/dr) of the cosine cutoff."""
    out = np.zeros(2)
    lib().orc_cutoff(float(r), float(rc), _ptr(out))
    return out[0], out[1]


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Packed:
    """Keeps the numpy buffers of a model alive while the C struct points at them."""

    def __init__(self, model):
        self.tw = _f64(model.type_weights)
        self.widths = np.ascontiguousarray(model.widths, dtype=np.int32)
        self.params = _f64(model.params)
        self.shift = None if model.in_shift is None else _f64(model.in_shift)
        self.scale = None if model.in_scale is None else _f64(model.in_scale)
        dp = C.POINTER(C.c_double)
        self.s = _Model(
            model.n_species, self.tw.ctypes.data_as(dp), float(model.rc_rad), int(model.order_rad),
            float(model.rc_ang), int(model.order_ang), len(model.widths) - 1,
            self.widths.ctypes.data_as(C.POINTER(C.c_int)), self.params.ctypes.data_as(dp),
            None if self.shift is None else self.shift.ctypes.data_as(dp),
            None if self.scale is None else self.scale.ctypes.data_as(dp))


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def compute(model, pos, types, box, mode=CELLS, n_threads=0, center_mask=None,
            want_G=False, want_dEdG=False, want_dEdW=False, want_forces=True):
    """Energy, forces [N,3], virial [3,3], per-atom energies, and optionally
    G / dE/dG [N,D] and dE/dW [n_species, n_params] of one structure."""
    pk = _Packed(model)
    pos = _f64(pos)
    types = np.ascontiguousarray(types, dtype=np.int32)
    box = _f64(box)
    n = pos.shape[0]
    D = model.widths[0]
    e = np.zeros(1)
    ea = np.zeros(n)
    F = np.zeros((n, 3)) if want_forces else None
    W = np.zeros((3, 3)) if want_forces else None
    G = np.zeros((n, D)) if want_G else None
    dG = np.zeros((n, D)) if want_dEdG else None
    dW = np.zeros_like(pk.params) if want_dEdW else None
    mask = None if center_mask is None else np.ascontiguousarray(center_mask, dtype=np.uint8)
    rc = lib().orc_compute(C.byref(pk.s), n, _ptr(pos), _ptr(types), _ptr(box), mode, n_threads,
                           _ptr(mask), _ptr(e), _ptr(ea), _ptr(F), _ptr(W), _ptr(G), _ptr(dG), _ptr(dW))
    _check(rc, "orc_compute")
    out = dict(energy=float(e[0]), e_atom=ea, forces=F, virial=W)
    if want_G:
        out["G"] = G
    if want_dEdG:
        out["dEdG"] = dG
    if want_dEdW:
        out["dEdW"] = dW
    return out


def compute_tri(model, pos, types, box, tilt, n_threads=0, want_G=False):
    """Energy, forces, virial, per-atom energies (and optionally G) of one
    structure in the restricted triclinic cell a = (L_x, 0, 0), b = (xy, L_y, 0),
    c = (xz, yz, L_z): box = (L_x, L_y, L_z), tilt = (xy, xz, yz). Brute-force
    lattice images (zero tilt takes the orthorhombic brute-force path)."""
    pk = _Packed(model)
    pos = _f64(pos)
    types = np.ascontiguousarray(types, dtype=np.int32)
    box = _f64(box)
    tilt = _f64(tilt)
    n = pos.shape[0]
    e = np.zeros(1)
    ea = np.zeros(n)
    F = np.zeros((n, 3))
    W = np.zeros((3, 3))
    G = np.zeros((n, model.widths[0])) if want_G else None
    rc = lib().orc_compute_tri(C.byref(pk.s), n, _ptr(pos), _ptr(types), _ptr(box), _ptr(tilt), BRUTE,
                               n_threads, _ptr(e), _ptr(ea), _ptr(F), _ptr(W), _ptr(G))
    _check(rc, "orc_compute_tri")
    out = dict(energy=float(e[0]), e_atom=ea, forces=F, virial=W)
    if want_G:
        out["G"] = G
    return out


def md_tri(model, pos, vel, types, box, tilt, dt, n_steps, n_threads=0, thermostat=None):
    """Velocity Verlet (optionally Berendsen) in a restricted triclinic cell;
    returns (pos, vel, e_pot[n+1], e_kin[n+1])."""
    pk = _Packed(model)
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    types = np.ascontiguousarray(types, dtype=np.int32)
    box = _f64(box)
    tilt = _f64(tilt)
    mass = _f64(model.masses)
    ep = np.zeros(n_steps + 1)
    ek = np.zeros(n_steps + 1)
    T0, tau = (0.0, 0.0) if thermostat is None else (float(thermostat[0]), float(thermostat[1]))
    rc = lib().orc_md_tri(C.byref(pk.s), pos.shape[0], _ptr(pos), _ptr(vel), _ptr(types), _ptr(mass),
                          _ptr(box), _ptr(tilt), float(dt), int(n_steps), n_threads, _ptr(ep), _ptr(ek), T0, tau)
    _check(rc, "orc_md_tri")
    return pos, vel, ep, ek


def md_npt(model, pos, vel, types, box, tilt, dt, n_steps, barostat, thermostat=None, n_threads=0):
    """Velocity Verlet with the Berendsen barostat (see aenet_oracle.c):
    barostat = (P0 in bar, tau_P in ps, bulk modulus in bar, every K steps);
    optional thermostat = (T0 in K, tau_T in ps). Returns (pos, vel, e_pot,
    e_kin, box, tilt) with the final cell."""
    pk = _Packed(model)
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    types = np.ascontiguousarray(types, dtype=np.int32)
    box = _f64(box).copy()
    tilt = _f64(tilt).copy()
    mass = _f64(model.masses)
    ep = np.zeros(n_steps + 1)
    ek = np.zeros(n_steps + 1)
    T0, tau = (0.0, 0.0) if thermostat is None else (float(thermostat[0]), float(thermostat[1]))
    P0, tau_p, modulus, every = barostat
    rc = lib().orc_md_npt(C.byref(pk.s), pos.shape[0], _ptr(pos), _ptr(vel), _ptr(types), _ptr(mass),
                          _ptr(box), _ptr(tilt), float(dt), int(n_steps), n_threads, _ptr(ep), _ptr(ek), T0, tau,
                          float(P0), float(tau_p), float(modulus), int(every))
    _check(rc, "orc_md_npt")
    return pos, vel, ep, ek, box, tilt


def forces_subset(model, pos, types, box, targets, mode=CELLS, n_threads=0):
    """Forces [T,3] and atomic energies [T] on the target atoms only."""
    pk = _Packed(model)
    pos = _f64(pos)
    types = np.ascontiguousarray(types, dtype=np.int32)
    box = _f64(box)
    tg = np.ascontiguousarray(targets, dtype=np.int32)
    F = np.zeros((len(tg), 3))
    Ea = np.zeros(len(tg))
    rc = lib().orc_forces_subset(C.byref(pk.s), pos.shape[0], _ptr(pos), _ptr(types), _ptr(box),
                                 mode, n_threads, len(tg), _ptr(tg), _ptr(F), _ptr(Ea))
    _check(rc, "orc_forces_subset")
    return F, Ea


def md_nve(model, pos, vel, types, box, dt, n_steps, mode=CELLS, n_threads=0, thermostat=None):
    """Velocity-Verlet NVE; returns (pos, vel, e_pot[n+1], e_kin[n+1]). With
    thermostat = (T0 in K, tau in ps): the Berendsen thermostat (velocities
    scaled at the start of every step, see aenet_oracle.c)."""
    pk = _Packed(model)
    pos = _f64(pos).copy()
    vel = _f64(vel).copy()
    types = np.ascontiguousarray(types, dtype=np.int32)
    box = _f64(box)
    mass = _f64(model.masses)
    ep = np.zeros(n_steps + 1)
    ek = np.zeros(n_steps + 1)
    if thermostat is None:
        rc = lib().orc_md_nve(C.byref(pk.s), pos.shape[0], _ptr(pos), _ptr(vel), _ptr(types), _ptr(mass),
                              _ptr(box), float(dt), int(n_steps), mode, n_threads, _ptr(ep), _ptr(ek))
    else:
        rc = lib().orc_md_nvt(C.byref(pk.s), pos.shape[0], _ptr(pos), _ptr(vel), _ptr(types), _ptr(mass),
                              _ptr(box), float(dt), int(n_steps), mode, n_threads, _ptr(ep), _ptr(ek),
                              float(thermostat[0]), float(thermostat[1]))
    _check(rc, "orc_md_nvt" if thermostat is not None else "orc_md_nve")
    return pos, vel, ep, ek


def neighbour_lists(pos, box, rc, mode=BRUTE):
    """Per-atom sorted lists of (j, n_x, n_y, n_z) image-atoms within rc."""
    pos = _f64(pos)
    box = _f64(box)
    n = pos.shape[0]
    counts = np.zeros(n, dtype=np.int32)
    _check(lib().orc_neighbour_lists(mode, n, _ptr(pos), _ptr(box), float(rc), _ptr(counts),
                                     None, None, None), "orc_neighbour_lists")
    offs = np.zeros(n + 1, dtype=np.int64)
    offs[1:] = np.cumsum(counts)
    js = np.zeros(max(1, offs[-1]), dtype=np.int32)
    imgs = np.zeros((max(1, offs[-1]), 3), dtype=np.int32)
    _check(lib().orc_neighbour_lists(mode, n, _ptr(pos), _ptr(box), float(rc), _ptr(counts),
                                     _ptr(offs), _ptr(js), _ptr(imgs)), "orc_neighbour_lists")
    out = []
    for i in range(n):
        rows = [(int(js[k]), *map(int, imgs[k])) for k in range(offs[i], offs[i + 1])]
        out.append(sorted(rows))
    return out
