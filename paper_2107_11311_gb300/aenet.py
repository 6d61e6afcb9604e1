"""Python binding of ``libaenet_gpu.so`` (C ABI in ``include/aenet_gpu.h``).

Argument marshalling only: every step of the potential runs in the library's
CUDA kernels. torch supplies device memory and the current CUDA stream; numpy
arrays and CPU tensors are passed as host pointers (the library stages them).
There is no CPU fallback: if the library is missing or no GPU is present the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

AENET_FP32, AENET_BF16, AENET_BF16X3 = 0, 1, 2
AENET_MD_ASYNC, AENET_MD_CONTINUE, AENET_MD_TIMING, AENET_MD_TIMING_POTENTIAL = 1, 2, 4, 8
AENET_OPT_KEEP_ACTIVATIONS = 1
AENET_OPT_FUSED_NETWORK = 2
AENET_OPT_PIPELINE = 3
AENET_OPT_MD_LIST = 4
AENET_MD_LIST_AUTO, AENET_MD_LIST_OFF, AENET_MD_LIST_ON = 0, 1, 2
AENET_PATH_FUSED = 1
AENET_PATH_PIPELINED = 2
AENET_PATH_LIST = 4
AENET_BATCH_AUTOTUNE = 1
STAGES = ("kick_drift_bin", "cell_sort", "descriptor", "network", "forces", "kick_reductions")
PRECISIONS = {"fp32": AENET_FP32, "bf16": AENET_BF16, "bf16x3": AENET_BF16X3}

STATUS = {0: "AENET_OK", -1: "AENET_E_ARG", -2: "AENET_E_CUDA", -3: "AENET_E_CAPACITY",
          -4: "AENET_E_NONFINITE", -5: "AENET_E_OVERLAP", -6: "AENET_E_TIMEOUT", -7: "AENET_E_NOMEM",
          -8: "AENET_E_STATE"}


class AenetError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class ModelDesc(C.Structure):
    _fields_ = [("n_species", C.c_int), ("type_weight", C.c_void_p), ("mass", C.c_void_p),
                ("rc_rad", C.c_double), ("order_rad", C.c_int), ("rc_ang", C.c_double),
                ("order_ang", C.c_int), ("n_layers", C.c_int), ("widths", C.c_void_p),
                ("params", C.c_void_p), ("in_shift", C.c_void_p), ("in_scale", C.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the C-ABI library (building it with nvcc if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"{path} is missing: run paper_2107_11311_gb300.build.build()")
        _build.build()
    lib = C.CDLL(path)
    P, I, D = C.c_void_p, C.c_int, C.c_double
    lib.aenet_setup.argtypes = [C.POINTER(P), C.POINTER(ModelDesc), I, P]
    lib.aenet_set_stream.argtypes = [P, P]
    lib.aenet_compute.argtypes = [P, I, P, P, P, P, P, P, P]
    lib.aenet_compute_async.argtypes = [P, I, P, P, P, P, P, P, P]
    lib.aenet_descriptors.argtypes = [P, I, P, P, P, P]
    lib.aenet_compute_batch.argtypes = [P, I, P, P, P, P, P, P, P]
    lib.aenet_batch_prepare.argtypes = [P, I, P, P, P, P, P, P, P, I]
    lib.aenet_batch_run.argtypes = [P]
    lib.aenet_set_skin.argtypes = [P, D]
    lib.aenet_set_box_tilt.argtypes = [P, D, D, D]
    lib.aenet_set_barostat.argtypes = [P, D, D, D, I]
    lib.aenet_md_box.argtypes = [P, P, P]
    lib.aenet_set_thermostat.argtypes = [P, D, D]
    lib.aenet_md_list_builds.argtypes = [P, P]
    lib.aenet_batch_tuning.argtypes = [P, P, P, P, P, P]
    lib.aenet_set_option.argtypes = [P, I, I]
    lib.aenet_grad_weights.argtypes = [P, P]
    lib.aenet_set_params.argtypes = [P, P]
    lib.aenet_md_nve.argtypes = [P, I, P, P, P, P, D, I, P, P, I]
    lib.aenet_check.argtypes = [P]
    lib.aenet_neighbor_stats.argtypes = [P, P]
    lib.aenet_descriptors_noalloc.argtypes = [I, P, P, P, I, P, D, I, D, I, P, P]
    lib.aenet_md_stage_times.argtypes = [P, P, P, P]
    lib.aenet_last_error.argtypes = [P]
    lib.aenet_last_error.restype = C.c_char_p
    lib.aenet_destroy.argtypes = [P]
    lib.aenet_destroy.restype = None
    _lib = lib
    return lib


def _is_torch(x):
    try:
        import torch
        return isinstance(x, torch.Tensor)
    except ImportError:  # pragma: no cover
        return False


def _ptr(x):
    """Raw pointer of a contiguous numpy array or torch tensor (or None)."""
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return C.c_void_p(x.ctypes.data)


def _as(x, dtype):
    """numpy inputs are converted to contiguous arrays of the ABI's type; torch
    tensors must already have it (no hidden copies of device data)."""
    if x is None:
        return None
    if _is_torch(x):
        import torch
        want = {np.float64: torch.float64, np.int32: torch.int32, np.float32: torch.float32}[dtype]
        if x.dtype != want:
            raise TypeError(f"expected a {want} tensor, got {x.dtype}")
        return x
    return np.ascontiguousarray(x, dtype=dtype)


def _current_stream():
    import torch
    if torch.cuda.is_available():
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return None


NOALLOC_MAX_ATOMS = 16384


def descriptors_noalloc(model, pos, types, box, out, stream=None):
    """Descriptor through the allocation-free entry point (no context, no device
    allocation; for callers that cannot call cudaMalloc). ``pos`` [n, 3] float64,
    ``types`` [n] int32 and ``out`` [n, D] float32 must be contiguous CUDA tensors
    on the current device; at most NOALLOC_MAX_ATOMS atoms; orthorhombic boxes
    only. ``stream``: a torch.cuda.Stream or a raw cudaStream_t handle (default:
    torch's current stream)."""
    lib = load()
    import torch
    for name, x in (("pos", pos), ("types", types), ("out", out)):
        if not _is_torch(x) or x.device.type != "cuda":
            raise TypeError(f"{name} must be a CUDA tensor")
        if x.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} is on cuda:{x.device.index}, not on the current device "
                             f"cuda:{torch.cuda.current_device()}")
    pos, types, out = _as(pos, np.float64), _as(types, np.int32), _as(out, np.float32)
    n = int(pos.shape[0])
    if pos.dim() != 2 or pos.shape[1] != 3:
        raise ValueError(f"pos must have shape (n, 3), got {tuple(pos.shape)}")
    if types.numel() != n:
        raise ValueError(f"types holds {types.numel()} entries for {n} atoms")
    D = 2 * (int(model.order_rad) + int(model.order_ang) + 2)
    if tuple(out.shape) != (n, D):
        raise ValueError(f"out must have shape ({n}, {D}), got {tuple(out.shape)}")
    box = np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    tw = np.ascontiguousarray(model.type_weights, dtype=np.float64)
    if stream is None:
        st = _current_stream()
    elif hasattr(stream, "cuda_stream"):  # a torch.cuda.Stream
        st = C.c_void_p(stream.cuda_stream)
    else:
        st = C.c_void_p(int(stream)) if not isinstance(stream, C.c_void_p) else stream
    rc = lib.aenet_descriptors_noalloc(n, _ptr(pos), _ptr(types), _ptr(box), int(model.n_species),
                                       _ptr(tw), float(model.rc_rad), int(model.order_rad), float(model.rc_ang),
                                       int(model.order_ang), _ptr(out), st)
    if rc != 0:
        raise AenetError(rc, lib.aenet_last_error(None).decode())
    return out


class AenetGPU:
    """One library context: a model resident on the current GPU.

    ``model`` is a :class:`paper_2107_11311_gb300.inputs.Model`.
    """

    def __init__(self, model, precision="fp32", stream=None):
        self.lib = load()
        self.model = model
        self.D = int(model.widths[0])
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        keep = dict(
            tw=np.ascontiguousarray(model.type_weights, dtype=np.float64),
            mass=np.ascontiguousarray(model.masses, dtype=np.float64) if len(model.masses) else None,
            widths=np.ascontiguousarray(model.widths, dtype=np.int32),
            params=np.ascontiguousarray(model.params, dtype=np.float64),
            shift=np.ascontiguousarray(model.in_shift, dtype=np.float64),
            scale=np.ascontiguousarray(model.in_scale, dtype=np.float64))
        desc = ModelDesc(model.n_species, keep["tw"].ctypes.data,
                         None if keep["mass"] is None else keep["mass"].ctypes.data,
                         float(model.rc_rad), int(model.order_rad), float(model.rc_ang), int(model.order_ang),
                         len(model.widths) - 1, keep["widths"].ctypes.data, keep["params"].ctypes.data,
                         keep["shift"].ctypes.data, keep["scale"].ctypes.data)
        h = C.c_void_p()
        st = stream if stream is not None else _current_stream()
        rc = self.lib.aenet_setup(C.byref(h), C.byref(desc), self.precision, st)
        if rc != 0:
            raise AenetError(rc, self.lib.aenet_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.aenet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise AenetError(rc, self.lib.aenet_last_error(self.h).decode())

    def set_stream(self, stream):
        """Order the context's work on `stream` (a raw cudaStream_t handle);
        a no-op when it already is the context's stream."""
        if getattr(self, "_stream", None) == stream:
            return
        self._check(self.lib.aenet_set_stream(self.h, C.c_void_p(stream)))
        self._stream = stream

    def check(self):
        self._check(self.lib.aenet_check(self.h))

    @staticmethod
    def _box(box):
        return np.ascontiguousarray(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))

    def compute(self, pos, types, box, energy=None, forces=None, virial=None, e_atom=None):
        """Energy, forces, virial (and per-atom energies) of one structure.

        With numpy inputs and no output buffers, returns numpy results. Output
        buffers (numpy or torch, host or device) may be passed to avoid copies.
        """
        pos, types = _as(pos, np.float64), _as(types, np.int32)
        n = int(pos.shape[0])
        ret = energy is None and forces is None and virial is None and e_atom is None
        if ret:
            energy, forces, virial, e_atom = np.zeros(1), np.zeros((n, 3)), np.zeros((3, 3)), np.zeros(n)
        box = self._box(box)
        self._check(self.lib.aenet_compute(self.h, n, _ptr(pos), _ptr(types), _ptr(box), _ptr(energy),
                                           _ptr(forces), _ptr(virial), _ptr(e_atom)))
        if ret:
            return dict(energy=float(energy[0]), forces=forces, virial=virial, e_atom=e_atom)
        return None

    def compute_async(self, pos, types, box, energy=None, forces=None, virial=None, e_atom=None):
        """The evaluation enqueued on the context's stream without waiting:
        every array a CUDA tensor; errors are reported by the next check()."""
        pos, types = _as(pos, np.float64), _as(types, np.int32)
        box = self._box(box)
        self._check(self.lib.aenet_compute_async(self.h, int(pos.shape[0]), _ptr(pos), _ptr(types), _ptr(box),
                                                 _ptr(energy), _ptr(forces), _ptr(virial), _ptr(e_atom)))

    def compute_batch(self, atom_offset, pos, types, boxes, energies=None, forces=None, virials=None):
        """Energies [S], forces [N,3], virials [S,3,3] of S structures in one
        evaluation; atom_offset [S+1] int64 and boxes [S,3] are host arrays."""
        pos, types = _as(pos, np.float64), _as(types, np.int32)
        off = np.ascontiguousarray(atom_offset, dtype=np.int64)
        bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
        S = len(off) - 1
        ret = energies is None and forces is None and virials is None
        if ret:
            energies, forces, virials = np.zeros(S), np.zeros((int(off[-1]), 3)), np.zeros((S, 3, 3))
        self._check(self.lib.aenet_compute_batch(self.h, S, _ptr(off), _ptr(pos), _ptr(types), _ptr(bx),
                                                 _ptr(energies), _ptr(forces), _ptr(virials)))
        if ret:
            return dict(energies=energies, forces=forces, virials=virials)
        return None

    def batch_prepare(self, atom_offset, boxes, pos, types, energies=None, forces=None, virials=None,
                      autotune=True):
        """Fix a batch layout and its device buffers (torch CUDA tensors: pos
        [N,3] float64, types [N] int32, energies [S], forces [N,3], virials
        [S,3,3] float64), tune the potential launch on the current pos and
        capture the evaluation in a CUDA graph. Returns batch_tuning()."""
        off = np.ascontiguousarray(atom_offset, dtype=np.int64)
        bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(-1, 3)
        S = len(off) - 1
        self._batch_keep = (off, bx, pos, types, energies, forces, virials)
        self._check(self.lib.aenet_batch_prepare(self.h, S, _ptr(off), _ptr(bx), _ptr(pos), _ptr(types),
                                                 _ptr(energies), _ptr(forces), _ptr(virials),
                                                 AENET_BATCH_AUTOTUNE if autotune else 0))
        return self.batch_tuning()

    def batch_run(self):
        """Replay the prepared batch on the context's stream (asynchronous)."""
        self._check(self.lib.aenet_batch_run(self.h))

    def batch_tuning(self):
        p, t, g, k = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        ms = C.c_float()
        self._check(self.lib.aenet_batch_tuning(self.h, C.byref(p), C.byref(t), C.byref(g), C.byref(k),
                                                C.byref(ms)))
        return dict(persistent=bool(p.value), tile=t.value, ctas=g.value, kernels=k.value, ms=ms.value)

    def descriptors(self, pos, types, box, out=None):
        pos, types = _as(pos, np.float64), _as(types, np.int32)
        n = int(pos.shape[0])
        G = np.zeros((n, self.D), dtype=np.float32) if out is None else out
        box = self._box(box)
        self._check(self.lib.aenet_descriptors(self.h, n, _ptr(pos), _ptr(types), _ptr(box), _ptr(G)))
        return G

    def md_nve(self, pos, vel, types, box, dt, n_steps, e_pot=None, e_kin=None, flags=0):
        """Velocity Verlet in place on ``pos`` and ``vel`` (float64 arrays or
        tensors; numpy arrays must already be float64 and contiguous): NVE, or
        with set_thermostat / set_barostat the Berendsen NVT / NPT couplings
        (the cell a barostat run ends in: md_box())."""
        types = _as(types, np.int32)
        n = int(pos.shape[0])
        box = self._box(box)
        self._check(self.lib.aenet_md_nve(self.h, n, _ptr(pos), _ptr(vel), _ptr(types), _ptr(box),
                                          float(dt), int(n_steps), _ptr(e_pot), _ptr(e_kin), int(flags)))

    def set_skin(self, skin):
        """Verlet-list skin (A) for md_nve; 0 rebuilds the cell list every step."""
        self._check(self.lib.aenet_set_skin(self.h, float(skin)))

    def set_box_tilt(self, xy, xz, yz):
        """Tilt factors of the restricted triclinic cell a = (L_x, 0, 0),
        b = (xy, L_y, 0), c = (xz, yz, L_z) used by later single-structure calls
        (box = (L_x, L_y, L_z)); zeros restore the orthorhombic box."""
        self._check(self.lib.aenet_set_box_tilt(self.h, float(xy), float(xz), float(yz)))

    def set_barostat(self, P0, tau, modulus, every=1):
        """Berendsen barostat for md_nve: target P0 (bar), coupling time tau (ps),
        bulk modulus (bar), coupling after every `every` steps; tau <= 0 turns it
        off."""
        self._check(self.lib.aenet_set_barostat(self.h, float(P0), float(tau), float(modulus), int(every)))

    def md_box(self):
        """(edges [3], tilts [3]) of the cell the last md_nve call ended in."""
        box, tilt = np.zeros(3), np.zeros(3)
        self._check(self.lib.aenet_md_box(self.h, _ptr(box), _ptr(tilt)))
        return box, tilt

    def set_thermostat(self, T0, tau):
        """Berendsen thermostat for md_nve: target T0 (K), coupling time tau (ps);
        tau <= 0 turns it off (NVE)."""
        self._check(self.lib.aenet_set_thermostat(self.h, float(T0), float(tau)))

    def md_list_builds(self):
        """Verlet-list builds so far on this context."""
        out = np.zeros(1, dtype=np.int64)
        self._check(self.lib.aenet_md_list_builds(self.h, _ptr(out)))
        return int(out[0])

    def set_option(self, option, value):
        self._check(self.lib.aenet_set_option(self.h, int(option), int(value)))

    def fuse_network(self, on=True):
        """BF16 forms: run the tensor-core networks inside the fused potential
        kernel (default) or as the three-kernel path (descriptor kernel, network
        kernel, force kernel)."""
        self.set_option(AENET_OPT_FUSED_NETWORK, 1 if on else 0)

    def pipeline(self, on=True):
        """FP32 fused form: the pipelined potential kernel, or (default) the
        block-synchronous one."""
        self.set_option(AENET_OPT_PIPELINE, 1 if on else 0)

    def md_list(self, mode="auto"):
        """MD steps without a skin: "on" builds the exact neighbour list in every
        step and evaluates it with the list-driven potential kernel, "off" lets
        the fused kernel search the cells itself, "auto" (default) takes "on"
        except for the spherical-harmonic basis (angular order 6, radial 20)."""
        modes = {"auto": AENET_MD_LIST_AUTO, "off": AENET_MD_LIST_OFF, "on": AENET_MD_LIST_ON}
        self.set_option(AENET_OPT_MD_LIST, modes[mode])

    def keep_activations(self, on=True):
        """Keep per-atom activation records so that grad_weights() can follow."""
        self.set_option(AENET_OPT_KEEP_ACTIVATIONS, 1 if on else 0)

    def grad_weights(self, out=None):
        """dE/dW [n_species, n_params] (FP64) of the last evaluation."""
        if out is None:
            out = np.zeros((self.model.n_species, self.model.n_params))
        self._check(self.lib.aenet_grad_weights(self.h, _ptr(out)))
        return out

    def set_params(self, params):
        """Replace the network parameters ([n_species, n_params] float64): a
        CUDA tensor is converted and packed on the device, in stream order and
        without a host round trip; numpy arrays go through the host."""
        if _is_torch(params) and params.is_cuda:
            p = _as(params.contiguous(), np.float64)
            self._params_keep = p  # valid until the stream has read it
        else:
            p = np.ascontiguousarray(params, dtype=np.float64)
        self._check(self.lib.aenet_set_params(self.h, _ptr(p)))

    def neighbor_stats(self):
        """(entries within the largest cutoff, angular entries, angular pairs) of
        the last evaluation, summed over atoms."""
        out = np.zeros(3, dtype=np.int64)
        self._check(self.lib.aenet_neighbor_stats(self.h, _ptr(out)))
        return tuple(int(x) for x in out)

    def md_stage_times(self):
        """Per-stage device milliseconds of the last timed MD step (None for the
        stages AENET_MD_TIMING_POTENTIAL does not record), the number of kernel
        launches per MD step and whether the fused kernel ran."""
        ms = np.zeros(len(STAGES), dtype=np.float32)
        k = C.c_int(0)
        f = C.c_int(0)
        self._check(self.lib.aenet_md_stage_times(self.h, _ptr(ms), C.byref(k), C.byref(f)))
        vals = [None if np.isnan(v) else float(v) for v in ms]
        return dict(zip(STAGES, vals)), int(k.value), bool(f.value & 1)

    def md_path_flags(self):
        """Path flags of the last timed MD step: AENET_PATH_FUSED (1) when one
        fused kernel ran descriptor, network and forces, AENET_PATH_PIPELINED (2)
        when it was the pipelined form, AENET_PATH_LIST (4) when the step built
        the exact neighbour list and ran the list-driven kernel."""
        ms = np.zeros(len(STAGES), dtype=np.float32)
        f = C.c_int(0)
        self._check(self.lib.aenet_md_stage_times(self.h, _ptr(ms), None, C.byref(f)))
        return int(f.value)


def _energy_function():
    import torch

    class AenetEnergy(torch.autograd.Function):
        """E(positions, parameters) with a hand-written backward: dE/dr = -F from
        the force kernel, dE/dW from the weight-gradient kernel. Usage:
        ``E = AenetEnergy.apply(pos, params, gpu, types, box)`` with ``gpu`` an
        AenetGPU, ``pos`` [N,3] float64 and ``params`` [n_species, n_params]
        float64 tensors."""

        @staticmethod
        def forward(ctx, pos, params, gpu, types, box):
            """On CUDA tensors everything is enqueued on torch's current stream:
            the parameters are converted and packed on the device, the
            evaluation and dE/dW follow without a host round trip. The first
            call for a system size runs the synchronous evaluation (it sizes the
            neighbour lists); later calls do not wait, so device-side errors are
            reported by gpu.check(), which callers run now and then."""
            want_w = params.requires_grad
            dev = pos.device
            on_gpu = dev.type == "cuda" and params.is_cuda and types.is_cuda
            if on_gpu:
                h = torch.cuda.current_stream(dev).cuda_stream
                if h:  # torch's legacy default stream (handle 0) already orders the context's blocking stream
                    gpu.set_stream(h)
                gpu.set_params(params.detach())
            else:
                gpu.set_params(params.detach().cpu().numpy())
            gpu.keep_activations(want_w)
            E = torch.zeros(1, dtype=torch.float64, device=dev)
            F = torch.zeros_like(pos, dtype=torch.float64)
            p = pos.detach().contiguous()
            n = int(p.shape[0])
            if on_gpu and getattr(gpu, "_async_n", None) == n:
                gpu.compute_async(p, types, box, energy=E, forces=F)
            else:
                gpu.compute(p, types, box, energy=E, forces=F)
                gpu._async_n = n if on_gpu else None
            dW = None
            if want_w:
                dW = torch.zeros(params.shape, dtype=torch.float64, device=dev)
                gpu.grad_weights(out=dW)
            ctx.save_for_backward(F, dW if dW is not None else torch.zeros(0))
            ctx.want_w = want_w
            return E[0]

        @staticmethod
        def backward(ctx, gE):
            F, dW = ctx.saved_tensors
            gp = -F * gE
            gw = (dW * gE).to(dtype=torch.float64) if ctx.want_w else None
            return gp, gw, None, None, None

    return AenetEnergy


def energy_function():
    """The torch.autograd.Function class (built lazily so that torch stays optional)."""
    global _AENET_ENERGY
    try:
        return _AENET_ENERGY
    except NameError:
        _AENET_ENERGY = _energy_function()
        return _AENET_ENERGY
