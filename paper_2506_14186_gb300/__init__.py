"""GB300-native batched soft-contact rollouts with a discrete adjoint.

Python binding of the C ABI in ``include/dmx.h`` (library ``libdmx.so`` built
in-tree by ``paper_2506_14186_gb300._build``).  This module only marshals
arguments: every step of the rollout and of its adjoint runs in the library's
CUDA kernels.  PyTorch supplies device memory and the current CUDA stream.
There is no CPU fallback: without the compiled library, or without a CUDA
device, the calls raise.

Batched arrays use the library's structure-of-arrays layout: ``x0`` is
``[nx, B]``, ``ctrl`` is ``[NI, nu, B]``, ``T`` is ``[B]`` (float64 CUDA tensors).
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import workloads  # noqa: F401  (scene descriptions and seeded inputs)

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libdmx.so")

c_i32, c_f64, c_p = ctypes.c_int32, ctypes.c_double, ctypes.c_void_p

DMX_OK, DMX_ERR_INVALID, DMX_ERR_OOM, DMX_ERR_CUDA, DMX_NOT_READY, DMX_ERR_TIMEOUT, DMX_ERR_UNIMPLEMENTED = range(7)
ENV_STATUS = {0: "ok", 1: "max_steps", 2: "h_underflow", 3: "nonfinite", 4: "solver_noconv", 5: "row_overflow"}
FORMS = {"persistent": 0, "step": 1, "graph": 2}
# integration schemes: adaptive Dormand-Prince 5(4) and Tsitouras 5(4), fixed-step semi-implicit Euler
METHODS = {"dopri5": 0, "tsit5": 1, "euler": 2}
ADJOINT_MODES = {"reverse": 0, "tangent": 1, "recompute": 2}
_JOINT = {"free": 0, "hinge": 1}
_GEOM = {"sphere": 0, "capsule": 1, "box": 2}
_ACT = {"motor": 0, "position": 1}

# names of every entry point declared in include/dmx.h
ABI_SYMBOLS = ("dmx_create_model", "dmx_destroy_model", "dmx_model_dims", "dmx_rollout", "dmx_rollout_grad",
               "dmx_tape_free", "dmx_tape_read", "dmx_autotune", "dmx_set_lanes", "dmx_model_info", "dmx_server_create", "dmx_submit", "dmx_poll",
               "dmx_server_destroy", "dmx_eval_rhs", "dmx_rollout_static", "dmx_set_adjoint", "dmx_eval_rhs_vjp",
               "dmx_fp64_peak", "dmx_model_params", "dmx_rollout_grad_params", "dmx_rollout_grad_otd",
               "dmx_last_error")


class BodyDesc(ctypes.Structure):
    _fields_ = [("parent", c_i32), ("joint", c_i32), ("pos", c_f64 * 3), ("quat", c_f64 * 4), ("axis", c_f64 * 3),
                ("mass", c_f64), ("com", c_f64 * 3), ("inertia", c_f64 * 3), ("damping", c_f64)]


class GeomDesc(ctypes.Structure):
    _fields_ = [("type", c_i32), ("body", c_i32), ("pos", c_f64 * 3), ("quat", c_f64 * 4), ("size", c_f64 * 3)]


class PairDesc(ctypes.Structure):
    _fields_ = [("geom1", c_i32), ("geom2", c_i32), ("condim", c_i32), ("mu", c_f64)]


class ActDesc(ctypes.Structure):
    _fields_ = [("type", c_i32), ("body", c_i32), ("gear", c_f64), ("kp", c_f64), ("kd", c_f64)]


class ModelDesc(ctypes.Structure):
    _fields_ = [("nbody", c_i32), ("ngeom", c_i32), ("npair", c_i32), ("nact", c_i32),
                ("body", ctypes.POINTER(BodyDesc)), ("geom", ctypes.POINTER(GeomDesc)),
                ("pair", ctypes.POINTER(PairDesc)), ("act", ctypes.POINTER(ActDesc)),
                ("gravity", c_f64 * 3), ("solref", c_f64 * 2), ("solimp", c_f64 * 5), ("solimp_cfd", c_f64 * 5),
                ("softplus", c_f64), ("qpos0", ctypes.POINTER(c_f64))]


class RolloutArgs(ctypes.Structure):
    _fields_ = [("B", c_i32), ("x0", c_p), ("ctrl", c_p), ("T", c_p), ("NI", c_i32), ("rtol", c_f64),
                ("atol", c_f64), ("h0", c_f64), ("max_steps", c_i32), ("K", c_i32), ("form", c_i32),
                ("lanes", c_i32), ("host", c_i32), ("xT", c_p), ("xb", c_p), ("nsteps", c_p), ("nrej", c_p),
                ("status", c_p), ("tape", ctypes.POINTER(c_p)), ("method", c_i32)]


class OtdArgs(ctypes.Structure):
    _fields_ = [("B", c_i32), ("NI", c_i32), ("xT", c_p), ("ctrl", c_p), ("T", c_p), ("rtol", c_f64), ("atol", c_f64),
                ("h0", c_f64), ("max_steps", c_i32), ("method", c_i32), ("cfd", c_i32), ("xT_bar", c_p),
                ("xb_bar", c_p), ("x0_bar", c_p), ("ctrl_bar", c_p), ("steps", c_p), ("status", c_p)]


class ServerCfg(ctypes.Structure):
    _fields_ = [("device_bytes", ctypes.c_int64), ("max_inflight", c_i32), ("nstreams", c_i32),
                ("host_stage_bytes", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("model", c_p), ("B", c_i32), ("NI", c_i32), ("max_steps", c_i32), ("K", c_i32), ("rtol", c_f64),
                ("atol", c_f64), ("h0", c_f64), ("x0", c_p), ("ctrl", c_p), ("T", c_p), ("grad", c_i32),
                ("cfd", c_i32), ("xT_bar", c_p), ("xT", c_p), ("x0_bar", c_p), ("ctrl_bar", c_p), ("status", c_p)]


_lib = None


class DmxError(RuntimeError):
    pass


def lib():
    """Load libdmx.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"libdmx.so not built ({_LIB_PATH}); run paper_2506_14186_gb300._build.build()")
        L = ctypes.CDLL(_LIB_PATH)
        L.dmx_last_error.restype = ctypes.c_char_p
        L.dmx_server_destroy.argtypes = [c_p, c_f64]
        for name in ("dmx_create_model", "dmx_model_dims", "dmx_rollout", "dmx_rollout_grad", "dmx_autotune",
                     "dmx_server_create", "dmx_submit", "dmx_poll", "dmx_server_destroy", "dmx_model_info",
                     "dmx_set_lanes", "dmx_eval_rhs", "dmx_tape_read", "dmx_rollout_static", "dmx_set_adjoint",
                     "dmx_eval_rhs_vjp", "dmx_fp64_peak", "dmx_model_params", "dmx_rollout_grad_params",
                     "dmx_rollout_grad_otd"):
            getattr(L, name).restype = c_i32
        L.dmx_destroy_model.restype = None
        L.dmx_tape_free.restype = None
        _lib = L
    return _lib


def _check(rc):
    if rc != DMX_OK:
        raise DmxError(f"dmx error {rc}: {lib().dmx_last_error().decode()}")


def _stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return c_p(s.cuda_stream)


def _ptr(t):
    return c_p(t.data_ptr()) if t is not None else c_p(0)


def _require_cuda(t, name, dtype=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}")


class Model:
    """A compiled model on the current CUDA device (from a workloads scene dict)."""

    def __init__(self, scene):
        L = lib()
        bodies = (BodyDesc * len(scene["bodies"]))()
        for i, b in enumerate(scene["bodies"]):
            bodies[i] = BodyDesc(b["parent"], _JOINT[b["joint"]], (c_f64 * 3)(*b["pos"]), (c_f64 * 4)(*b["quat"]),
                                 (c_f64 * 3)(*b["axis"]), b["mass"], (c_f64 * 3)(*b["com"]),
                                 (c_f64 * 3)(*b["inertia"]), b["damping"])
        geoms = (GeomDesc * max(1, len(scene["geoms"])))()
        for i, g in enumerate(scene["geoms"]):
            geoms[i] = GeomDesc(_GEOM[g["type"]], g["body"], (c_f64 * 3)(*g["pos"]), (c_f64 * 4)(*g["quat"]),
                                (c_f64 * 3)(*g["size"]))
        pairs = (PairDesc * max(1, len(scene["pairs"])))()
        for i, p in enumerate(scene["pairs"]):
            pairs[i] = PairDesc(p["geom1"], p["geom2"], p["condim"], p["mu"])
        acts = (ActDesc * max(1, len(scene["actuators"])))()
        for i, a in enumerate(scene["actuators"]):
            acts[i] = ActDesc(_ACT[a["type"]], a["body"], a["gear"], a["kp"], a["kd"])
        o = scene["options"]
        q0 = (c_f64 * len(scene["qpos0"]))(*scene["qpos0"])
        desc = ModelDesc(len(scene["bodies"]), len(scene["geoms"]), len(scene["pairs"]), len(scene["actuators"]),
                         bodies, geoms, pairs, acts, (c_f64 * 3)(*o["gravity"]), (c_f64 * 2)(*o["solref"]),
                         (c_f64 * 5)(*o["solimp"]), (c_f64 * 5)(*o["solimp_cfd"]), o["softplus"], q0)
        h = c_p()
        _check(L.dmx_create_model(ctypes.byref(desc), ctypes.byref(h)))
        self.h = h
        self.scene = scene
        nq, nv, nu = c_i32(), c_i32(), c_i32()
        _check(L.dmx_model_dims(h, ctypes.byref(nq), ctypes.byref(nv), ctypes.byref(nu)))
        self.nq, self.nv, self.nu = nq.value, nv.value, nu.value
        self.nx = self.nq + self.nv

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().dmx_destroy_model(self.h)
        except Exception:
            pass

    def info(self):
        invw = (c_f64 * 16)()
        info = (c_i32 * 8)()
        _check(lib().dmx_model_info(self.h, invw, info))
        return {"invw": list(invw)[:info[5]], "nslot": info[0], "nrowid": info[1], "rcap": info[2],
                "ws_doubles": info[3], "ws_ints": info[4]}

    def lanes(self, B, grad=False):
        out = c_i32()
        _check(lib().dmx_autotune(self.h, int(B), int(grad), ctypes.byref(out), c_p(0)))
        return out.value

    def set_lanes(self, B, lanes, grad=False):
        """grad: False / 0 forward rollout, True / 1 taped rollout, 2 reverse-mode adjoint kernel."""
        _check(lib().dmx_set_lanes(self.h, int(B), int(grad), int(lanes)))

    def params(self):
        """Model parameters of rollout_grad_params: numpy array of t_c, phi_d,
        d_o, d_w, width, midpoint, mu of every pair, the mass of every body, then the side
        length of every box geom."""
        n = c_i32()
        _check(lib().dmx_model_params(self.h, ctypes.byref(n), None))
        vals = (c_f64 * n.value)()
        _check(lib().dmx_model_params(self.h, ctypes.byref(n), vals))
        return np.array(list(vals))

    def set_adjoint(self, mode):
        """Adjoint kernel of rollout_grad: "reverse" (default; stage snapshots in
        device memory when they fit), "recompute" (reverse mode evaluating each
        stage's right-hand side again) or "tangent" (forward-mode columns)."""
        _check(lib().dmx_set_adjoint(self.h, ADJOINT_MODES[mode]))


class Tape:
    """Checkpoints + accepted step sizes of one taped rollout (library owned)."""

    def __init__(self, handle, model, B, NI):
        self.h, self.model, self.B, self.NI = handle, model, B, NI

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().dmx_tape_free(self.h)
        except Exception:
            pass

    def read(self, stream=None, checkpoints=False):
        """(hlog [max_steps, B], nsteps [B]) as CUDA tensors, plus the
        checkpoints [ncheck, nx+1, B] when checkpoints=True."""
        import torch
        dims = (c_i32 * 6)()
        _check(lib().dmx_tape_read(self.h, None, None, None, dims, c_p(0)))
        hlog = torch.empty((dims[2], self.B), dtype=torch.float64, device="cuda")
        n = torch.empty(self.B, dtype=torch.int32, device="cuda")
        ck = torch.empty((dims[4], dims[5] + 1, self.B), dtype=torch.float64, device="cuda") if checkpoints else None
        _check(lib().dmx_tape_read(self.h, _ptr(hlog), _ptr(n), _ptr(ck), dims, _stream_handle(stream)))
        return (hlog, n, ck) if checkpoints else (hlog, n)


def rollout(model, x0, T, ctrl=None, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000, K=32,
            form="persistent", lanes=0, want_xb=False, tape=False, stream=None, method="dopri5"):
    """Batched rollout on the device (method: "dopri5" / "tsit5" adaptive, "euler"
    fixed step h0).  Returns a dict of CUDA tensors xT [nx, B], xb [NI+1, nx, B]
    (if want_xb), nsteps/nrej/status [B] (int32) and, with tape=True, a Tape for
    rollout_grad."""
    import torch
    _require_cuda(x0, "x0", torch.float64)
    _require_cuda(T, "T", torch.float64)
    B = x0.shape[1]
    if x0.shape[0] != model.nx or T.shape != (B,):
        raise ValueError("x0 must be [nx, B] and T [B]")
    if model.nu:
        if ctrl is None:
            raise ValueError("ctrl [NI, nu, B] required")
        _require_cuda(ctrl, "ctrl", torch.float64)
        if tuple(ctrl.shape) != (NI, model.nu, B):
            raise ValueError("ctrl must be [NI, nu, B]")
    dev = x0.device
    xT = torch.empty((model.nx, B), dtype=torch.float64, device=dev)
    xb = torch.empty((NI + 1, model.nx, B), dtype=torch.float64, device=dev) if want_xb else None
    nsteps = torch.empty(B, dtype=torch.int32, device=dev)
    nrej = torch.empty(B, dtype=torch.int32, device=dev)
    status = torch.empty(B, dtype=torch.int32, device=dev)
    th = c_p()
    args = RolloutArgs(B, x0.data_ptr(), ctrl.data_ptr() if (model.nu and ctrl is not None) else None, T.data_ptr(),
                       NI, rtol, atol, h0, max_steps, K, FORMS[form], lanes, 0, xT.data_ptr(),
                       xb.data_ptr() if xb is not None else None, nsteps.data_ptr(), nrej.data_ptr(),
                       status.data_ptr(), ctypes.pointer(th) if tape else None, METHODS[method])
    _check(lib().dmx_rollout(model.h, ctypes.byref(args), _stream_handle(stream)))
    out = {"xT": xT, "xb": xb, "nsteps": nsteps, "nrej": nrej, "status": status}
    if tape:
        out["tape"] = Tape(th, model, B, NI)
    return out


def rollout_host(model, x0, T, ctrl=None, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000, form="persistent",
                 lanes=0, xT=None, stream=None, method="dopri5"):
    """Same rollout through the C ABI with HOST buffers (numpy arrays or pinned
    CPU tensors, SoA layout); the library copies in, integrates and copies out."""
    def host_ptr(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return a.data_ptr()
        return a.ctypes.data
    B = x0.shape[1]
    if xT is None:
        xT = np.empty((model.nx, B))
    status = np.empty(B, dtype=np.int32)
    nsteps = np.empty(B, dtype=np.int32)
    args = RolloutArgs(B, host_ptr(x0), host_ptr(ctrl) if model.nu else None, host_ptr(T), NI, rtol, atol, h0,
                       max_steps, 32, FORMS[form], lanes, 1, host_ptr(xT), None, host_ptr(nsteps), None,
                       host_ptr(status), None, METHODS[method])
    _check(lib().dmx_rollout(model.h, ctypes.byref(args), _stream_handle(stream)))
    return {"xT": xT, "status": status, "nsteps": nsteps}


def rollout_grad(tape, xT_bar, xb_bar=None, cfd=False, stream=None):
    """Discrete adjoint of a taped rollout: returns (x0_bar [nx, B], ctrl_bar [NI, nu, B] or None)."""
    import torch
    m = tape.model
    _require_cuda(xT_bar, "xT_bar", torch.float64)
    if xb_bar is not None:
        _require_cuda(xb_bar, "xb_bar", torch.float64)
    x0_bar = torch.empty((m.nx, tape.B), dtype=torch.float64, device=xT_bar.device)
    ctrl_bar = torch.empty((tape.NI, m.nu, tape.B), dtype=torch.float64, device=xT_bar.device) if m.nu else None
    _check(lib().dmx_rollout_grad(m.h, tape.h, int(cfd), _ptr(xT_bar), _ptr(xb_bar), _ptr(x0_bar), _ptr(ctrl_bar),
                                  _stream_handle(stream)))
    return x0_bar, ctrl_bar


def rollout_grad_params(tape, xT_bar, xb_bar=None, cfd=False, stream=None):
    """Discrete adjoint with model-parameter gradients: returns (x0_bar [nx, B],
    ctrl_bar [NI, nu, B] or None, p_bar [np, B], p_bar_sum [np])."""
    import torch
    m = tape.model
    _require_cuda(xT_bar, "xT_bar", torch.float64)
    if xb_bar is not None:
        _require_cuda(xb_bar, "xb_bar", torch.float64)
    npar = len(m.params())
    dev = xT_bar.device
    x0_bar = torch.empty((m.nx, tape.B), dtype=torch.float64, device=dev)
    ctrl_bar = torch.empty((tape.NI, m.nu, tape.B), dtype=torch.float64, device=dev) if m.nu else None
    p_bar = torch.empty((npar, tape.B), dtype=torch.float64, device=dev)
    p_sum = torch.empty(npar, dtype=torch.float64, device=dev)
    _check(lib().dmx_rollout_grad_params(m.h, tape.h, int(cfd), _ptr(xT_bar), _ptr(xb_bar), _ptr(x0_bar),
                                         _ptr(ctrl_bar), _ptr(p_bar), _ptr(p_sum), _stream_handle(stream)))
    return x0_bar, ctrl_bar, p_bar, p_sum


def rollout_grad_otd(model, xT, T, xT_bar, ctrl=None, NI=1, xb_bar=None, cfd=False, rtol=1e-6, atol=1e-8, h0=1e-3,
                     max_steps=20000, method="dopri5", stream=None):
    """Optimize-then-discretize gradient (backsolve) from the final states xT
    [nx, B]: returns (x0_bar [nx, B], ctrl_bar [NI, nu, B] or None, steps [B],
    status [B]) of the backward solve."""
    import torch
    for t_, nm in ((xT, "xT"), (T, "T"), (xT_bar, "xT_bar")):
        _require_cuda(t_, nm, torch.float64)
    B = xT.shape[1]
    dev = xT.device
    x0_bar = torch.empty((model.nx, B), dtype=torch.float64, device=dev)
    ctrl_bar = torch.empty((NI, model.nu, B), dtype=torch.float64, device=dev) if model.nu else None
    steps = torch.empty(B, dtype=torch.int32, device=dev)
    status = torch.empty(B, dtype=torch.int32, device=dev)
    if model.nu:
        _require_cuda(ctrl, "ctrl", torch.float64)
    args = OtdArgs(B, NI, xT.data_ptr(), ctrl.data_ptr() if model.nu else None, T.data_ptr(), rtol, atol, h0,
                   max_steps, METHODS[method], int(cfd), xT_bar.data_ptr(),
                   xb_bar.data_ptr() if xb_bar is not None else None, x0_bar.data_ptr(),
                   ctrl_bar.data_ptr() if ctrl_bar is not None else None, steps.data_ptr(), status.data_ptr())
    _check(lib().dmx_rollout_grad_otd(model.h, ctypes.byref(args), _stream_handle(stream)))
    return x0_bar, ctrl_bar, steps, status


def eval_rhs_vjp(model, q, v, abar, u=None, cfd=False, lanes=0, stream=None):
    """Vector-Jacobian product of the right-hand side at B states: returns
    (qbar [nq, B], vbar [nv, B], ubar [nu, B] or None, status [B] int32)."""
    import torch
    for t, nm in ((q, "q"), (v, "v"), (abar, "abar")):
        _require_cuda(t, nm, torch.float64)
    B = q.shape[1]
    qbar = torch.empty((model.nq, B), dtype=torch.float64, device=q.device)
    vbar = torch.empty((model.nv, B), dtype=torch.float64, device=q.device)
    ubar = torch.empty((model.nu, B), dtype=torch.float64, device=q.device) if model.nu else None
    status = torch.empty(B, dtype=torch.int32, device=q.device)
    if model.nu:
        _require_cuda(u, "u", torch.float64)
    _check(lib().dmx_eval_rhs_vjp(model.h, B, _ptr(q), _ptr(v), _ptr(u) if model.nu else c_p(0), _ptr(abar), int(cfd),
                                  int(lanes), _ptr(qbar), _ptr(vbar), _ptr(ubar), _ptr(status),
                                  _stream_handle(stream)))
    return qbar, vbar, ubar, status


def eval_rhs(model, q, v, u=None, cfd=False, lanes=0, stream=None):
    """Right-hand side v' = F(q, v, u) for B states (q [nq, B], v [nv, B], u [nu, B]);
    returns (a [nv, B], info [4, B] int32: status, rows, active rows, 0)."""
    import torch
    _require_cuda(q, "q", torch.float64)
    _require_cuda(v, "v", torch.float64)
    B = q.shape[1]
    a = torch.empty((model.nv, B), dtype=torch.float64, device=q.device)
    info = torch.empty((4, B), dtype=torch.int32, device=q.device)
    if model.nu:
        _require_cuda(u, "u", torch.float64)
    _check(lib().dmx_eval_rhs(model.h, B, _ptr(q), _ptr(v), _ptr(u) if model.nu else c_p(0), int(cfd), int(lanes),
                              _ptr(a), _ptr(info), _stream_handle(stream)))
    return a, info


def rollout_static(model, x0, T, ctrl=None, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000, lanes=0,
                   xT=None, nsteps=None, status=None, stream=None, method="dopri5"):
    """dmx_rollout_static: the rollout without any device allocation inside
    the call (state in the library's fixed device array).  Outputs go to the
    caller's tensors xT [nx, B], nsteps / status [B] (int32); allocate them
    up front if this call must not allocate either.  Returns (xT, nsteps, status)."""
    import torch
    _require_cuda(x0, "x0", torch.float64)
    _require_cuda(T, "T", torch.float64)
    B = x0.shape[1]
    if model.nu:
        _require_cuda(ctrl, "ctrl", torch.float64)
    if xT is None:
        xT = torch.empty((model.nx, B), dtype=torch.float64, device=x0.device)
    if nsteps is None:
        nsteps = torch.empty(B, dtype=torch.int32, device=x0.device)
    if status is None:
        status = torch.empty(B, dtype=torch.int32, device=x0.device)
    args = RolloutArgs(B, x0.data_ptr(), ctrl.data_ptr() if model.nu else None, T.data_ptr(), NI, rtol, atol, h0,
                       max_steps, 1, FORMS["step"], lanes, 0, xT.data_ptr(), None, nsteps.data_ptr(), None,
                       status.data_ptr(), None, METHODS[method])
    _check(lib().dmx_rollout_static(model.h, ctypes.byref(args), _stream_handle(stream)))
    return xT, nsteps, status


def fp64_peak(configs=((4, 512), (8, 256), (2, 1024), (16, 128)), iters=8192, reps=3, stream=None):
    """Measured FP64 throughput of this GPU (TFLOP/s): the DFMA probe kernel
    timed with CUDA events on the stream, best over launch shapes (blocks per
    SM, threads) and repetitions.  Returns (tflops, {shape: tflops})."""
    import torch
    dev = torch.cuda.current_device()
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    h = _stream_handle(st)
    res = {}
    for per_sm, threads in configs:
        blocks = per_sm * nsm
        _check(lib().dmx_fp64_peak(blocks, threads, iters, _ptr(sink), h))      # warm-up
        best = 0.0
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _check(lib().dmx_fp64_peak(blocks, threads, iters, _ptr(sink), h))
            e1.record(st)
            e1.synchronize()
            best = max(best, 16.0 * blocks * threads * iters / (e0.elapsed_time(e1) * 1e-3) / 1e12)
        res[f"{per_sm}x{threads}"] = best
    return max(res.values()), res


def _rollout_fn_class():
    import torch

    class RolloutFn(torch.autograd.Function):
        """(x0 [nx, B], ctrl [NI, nu, B] or None) -> (xT [nx, B], xb [NI+1, nx, B]).
        Forward: taped dmx_rollout; backward: dmx_rollout_grad (discrete adjoint
        over the accepted steps, straight-through CFD when cfd=True)."""

        @staticmethod
        def forward(ctx, x0, ctrl, model, T, opts):
            o = dict(opts)
            cfd = o.pop("cfd", False)
            out = rollout(model, x0.detach(), T, ctrl=None if ctrl is None else ctrl.detach(), tape=True,
                          want_xb=True, **o)
            ctx.tape, ctx.cfd, ctx.has_ctrl = out["tape"], cfd, ctrl is not None
            ctx.mark_non_differentiable(out["status"])
            return out["xT"], out["xb"], out["status"]

        @staticmethod
        def backward(ctx, xT_bar, xb_bar, _status_bar):
            import torch as th
            if xT_bar is None:
                xT_bar = th.zeros((ctx.tape.model.nx, ctx.tape.B), dtype=th.float64, device="cuda")
            x0_bar, ctrl_bar = rollout_grad(ctx.tape, xT_bar.contiguous(),
                                            None if xb_bar is None else xb_bar.contiguous(), cfd=ctx.cfd)
            return x0_bar, (ctrl_bar if ctx.has_ctrl else None), None, None, None

    return RolloutFn


_RolloutFn = None


def rollout_fn(model, x0, T, ctrl=None, **opts):
    """Differentiable rollout: returns (xT, xb, status); gradients of any loss of
    xT / xb flow to x0 and ctrl through the library's adjoint kernel."""
    global _RolloutFn
    if _RolloutFn is None:
        _RolloutFn = _rollout_fn_class()
    return _RolloutFn.apply(x0, ctrl, model, T, opts)


class Server:
    """Continuous-batching request server (dmx_server_*): requests of any
    model, batch size and horizon are queued by submit() and admitted to the
    device as slots and memory free up; poll() returns the outputs (host
    arrays) and the submit-to-completion latency once a request is done."""

    def __init__(self, device_bytes=8 << 30, max_inflight=8, nstreams=8, host_stage_bytes=0):
        cfg = ServerCfg(int(device_bytes), int(max_inflight), int(nstreams), int(host_stage_bytes))
        h = c_p()
        _check(lib().dmx_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h
        self._live = {}

    @staticmethod
    def _host(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        return a

    def submit(self, model, x0, T, ctrl=None, NI=1, grad=False, xT_bar=None, cfd=False, rtol=1e-6, atol=1e-8,
               h0=1e-3, max_steps=20000, K=32):
        """x0 [nx, B], T [B], ctrl [NI, nu, B], xT_bar [nx, B] (host arrays, SoA).
        Returns a ticket."""
        x0 = self._host(x0); T = self._host(T)
        B = x0.shape[1]
        keep = {"x0": x0, "T": T, "model": model}
        keep["xT"] = np.empty((model.nx, B))
        keep["status"] = np.empty(B, dtype=np.int32)
        if model.nu:
            keep["ctrl"] = self._host(ctrl)
        if grad:
            keep["xT_bar"] = self._host(xT_bar)
            keep["x0_bar"] = np.empty((model.nx, B))
            keep["ctrl_bar"] = np.empty((NI, model.nu, B)) if model.nu else None
        ptr = lambda k: keep[k].ctypes.data if keep.get(k) is not None else None
        req = Request(model.h.value, B, NI, max_steps, K, rtol, atol, h0, ptr("x0"), ptr("ctrl"), ptr("T"), int(grad),
                      int(cfd), ptr("xT_bar"), ptr("xT"), ptr("x0_bar"), ptr("ctrl_bar"), ptr("status"))
        t = ctypes.c_uint64()
        _check(lib().dmx_submit(self.h, ctypes.byref(req), ctypes.byref(t)))
        self._live[t.value] = keep
        return t.value

    def poll(self, ticket):
        """None while the request runs; else a dict of its outputs and latency_s."""
        lat = c_f64()
        rc = lib().dmx_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(lat))
        if rc == DMX_NOT_READY:
            return None
        keep = self._live.pop(ticket, None)
        _check(rc)
        out = {k: keep[k] for k in ("xT", "status", "x0_bar", "ctrl_bar") if keep.get(k) is not None}
        out["latency_s"] = lat.value
        return out

    def wait(self, ticket, timeout=600.0, sleep=1e-4):
        import time
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError(f"request {ticket} not done after {timeout} s")
            time.sleep(sleep)

    def close(self, timeout=600.0):
        if getattr(self, "h", None):
            _check(lib().dmx_server_destroy(self.h, c_f64(timeout)))
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
