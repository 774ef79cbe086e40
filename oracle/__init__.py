"""CPU oracle of the batched soft-contact rollout and its discrete adjoint.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow FP64 restatement of
the method of arXiv 2506.14186 (DiffMJX + contacts from distance) written in
C++ (``oracle/*.h``, ``oracle/*.cpp``) and loaded through ctypes.  Only the
tests, the package smoke check and the CPU-baseline leg of the benchmark may
import it; the product path never does.

It shares no code with the CUDA path: scenes arrive as the plain dicts of
``paper_2506_14186_gb300.workloads`` and are packed here into the oracle's own
flat record layout (``oracle/model.h``).

Functions whose results are pinned by tests against closed forms, invariants,
brute force or finite differences (see ``tests/test_oracle_*.py``):
kinematics, mass matrix, bias force, contacts, impedance, constraint solve,
right-hand side and its Jacobian, DOPRI5 tableau, error norm and PID
step-size controller (fixed point, gains, rejection, clips and floor;
``tests/test_oracle_step_control.py``), rollout, replay, step Jacobian and
rollout gradient.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liborc.so")
_SRC = ["capi.cpp", "model.cpp"]
_HDR = ["scalar.h", "model.h", "dynamics.h", "integrator.h"]
_lib = None

JOINT = {"free": 0, "hinge": 1}
GEOM = {"sphere": 0, "capsule": 1, "box": 2}
ACT = {"motor": 0, "position": 1}
STATUS = {0: "ok", 1: "max_steps", 2: "h_underflow", 3: "nonfinite", 4: "solver_noconv"}
# integration schemes: adaptive Dormand-Prince 5(4) and Tsitouras 5(4), fixed-step semi-implicit Euler
METHODS = {"dopri5": 0, "tsit5": 1, "euler": 2}


def build(force: bool = False) -> str:
    """Compile liborc.so with g++ (-O2, no FMA contraction so x86 and Arm agree)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    deps = srcs + [os.path.join(_HERE, h) for h in _HDR]
    if not force and os.path.exists(_SO) and all(os.path.getmtime(_SO) >= os.path.getmtime(d) for d in deps):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared", "-pthread", *srcs, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_free.argtypes = [ctypes.c_void_p]
        L.orc_body_invw.restype = ctypes.c_double
        L.orc_pair_invw.restype = ctypes.c_double
        L.orc_impedance.restype = ctypes.c_double
        L.orc_count_flops.restype = ctypes.c_longlong
        L.orc_count_adjoint_flops.restype = ctypes.c_longlong
        L.orc_step_error.restype = ctypes.c_double
        L.orc_error_norm.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def pack_scene(scene):
    """Scene dict -> the oracle's flat records (body 20, geom 12, pair 4, act 5, opt 16)."""
    body = []
    for b in scene["bodies"]:
        body += [b["parent"], JOINT[b["joint"]], *b["pos"], *b["quat"], *b["axis"], b["mass"], *b["com"],
                 *b["inertia"], b["damping"]]
    geom = []
    for g in scene["geoms"]:
        geom += [GEOM[g["type"]], g["body"], *g["pos"], *g["quat"], *g["size"]]
    pair = []
    for p in scene["pairs"]:
        pair += [p["geom1"], p["geom2"], p["condim"], p["mu"]]
    act = []
    for a in scene["actuators"]:
        act += [ACT[a["type"]], a["body"], a["gear"], a["kp"], a["kd"]]
    o = scene["options"]
    opt = [*o["gravity"], *o["solref"], *o["solimp"], *o["solimp_cfd"], o["softplus"]]
    return (_f64(body), len(scene["bodies"]), _f64(geom if geom else [0.0]), len(scene["geoms"]),
            _f64(pair if pair else [0.0]), len(scene["pairs"]), _f64(act if act else [0.0]),
            len(scene["actuators"]), _f64(opt), _f64(scene["qpos0"]))


class OracleModel:
    """One compiled oracle model (single-environment and batched calls)."""

    def __init__(self, scene):
        L = lib()
        self._keep = pack_scene(scene)
        body, nb, geom, ng, pair, npair, act, na, opt, q0 = self._keep
        err = ctypes.create_string_buffer(256)
        h = L.orc_create(_p(body), nb, _p(geom), ng, _p(pair), npair, _p(act), na, _p(opt), _p(q0), err, 256)
        if not h:
            raise ValueError("oracle model: " + err.value.decode())
        self.h = ctypes.c_void_p(h)
        d = np.zeros(6, dtype=np.int32)
        L.orc_dims(self.h, _p(d))
        self.nq, self.nv, self.nu, self.nslot, self.nrowmax, self.nbody = (int(x) for x in d)
        self.nx = self.nq + self.nv

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().orc_free(self.h)
        except Exception:
            pass

    # ---------------------------------------------------------------- pieces
    def body_invw(self, b):
        return lib().orc_body_invw(self.h, b)

    def pair_invw(self, p):
        return lib().orc_pair_invw(self.h, p)

    def kinematics(self, q):
        R = np.zeros((self.nbody, 3, 3)); p = np.zeros((self.nbody, 3)); c = np.zeros((self.nbody, 3))
        lib().orc_kinematics(self.h, _p(_f64(q)), _p(R), _p(p), _p(c))
        return R, p, c

    def point_jacobian(self, q, body, x):
        Jl = np.zeros((3, self.nv)); Ja = np.zeros((3, self.nv))
        lib().orc_point_jacobian(self.h, _p(_f64(q)), int(body), _p(_f64(x)), _p(Jl), _p(Ja))
        return Jl, Ja

    def mass(self, q):
        M = np.zeros((self.nv, self.nv))
        lib().orc_mass(self.h, _p(_f64(q)), _p(M))
        return M

    def bias(self, q, v):
        c = np.zeros(self.nv)
        lib().orc_bias(self.h, _p(_f64(q)), _p(_f64(v)), _p(c))
        return c

    def applied(self, q, v, u=None):
        t = np.zeros(self.nv)
        u = _f64(u if u is not None else np.zeros(max(self.nu, 1)))
        lib().orc_applied(self.h, _p(_f64(q)), _p(_f64(v)), _p(u), _p(t))
        return t

    def contacts(self, q):
        out = np.zeros((self.nslot, 16))
        lib().orc_contacts(self.h, _p(_f64(q)), _p(out))
        return out

    def impedance(self, r, cfd=False):
        return lib().orc_impedance(self.h, ctypes.c_double(r), int(cfd))

    def rows(self, q, v, cfd=False):
        J = np.zeros((max(self.nrowmax, 1), self.nv)); aref = np.zeros(max(self.nrowmax, 1))
        D = np.zeros(max(self.nrowmax, 1)); slot = np.zeros(max(self.nrowmax, 1), dtype=np.int32)
        nr = lib().orc_rows(self.h, _p(_f64(q)), _p(_f64(v)), int(cfd), _p(J), _p(aref), _p(D), _p(slot))
        return J[:nr], aref[:nr], D[:nr], slot[:nr]

    def rhs(self, q, v, u=None, cfd=False, detail=False):
        a = np.zeros(self.nv); f = np.zeros(max(self.nrowmax, 1)); act = np.zeros(max(self.nrowmax, 1), dtype=np.int32)
        info = np.zeros(4, dtype=np.int32)
        u = _f64(u if u is not None else np.zeros(max(self.nu, 1)))
        rc = lib().orc_rhs(self.h, _p(_f64(q)), _p(_f64(v)), _p(u), int(cfd), _p(a), _p(f), _p(act), _p(info))
        if not detail:
            return a
        nr = int(info[0])
        return a, {"f": f[:nr], "active": act[:nr].astype(bool), "nr": nr, "iters": int(info[1]),
                   "noconv": bool(info[2]), "spd_fail": bool(info[3]), "rc": rc}

    def rhs_jacobian(self, q, v, u=None, cfd=False):
        Jq = np.zeros((self.nv, self.nq)); Jv = np.zeros((self.nv, self.nv)); Ju = np.zeros((self.nv, max(self.nu, 1)))
        u = _f64(u if u is not None else np.zeros(max(self.nu, 1)))
        lib().orc_rhs_jacobian(self.h, _p(_f64(q)), _p(_f64(v)), _p(u), int(cfd), _p(Jq), _p(Jv), _p(Ju))
        return Jq, Jv, Ju[:, :self.nu]

    def integrate_pos(self, q, dlt):
        out = np.zeros(self.nq)
        lib().orc_integrate_pos(self.h, _p(_f64(q)), _p(_f64(dlt)), _p(out))
        return out

    def step_error(self, x, h, u=None, rtol=1e-6, atol=1e-8, method="dopri5"):
        """Error norm of one attempt of size h from x (accepted iff <= 1; 0 for a fixed-step scheme)."""
        u = _f64(u if u is not None else np.zeros(max(self.nu, 1)))
        return lib().orc_step_error(self.h, _p(_f64(x)), _p(u), ctypes.c_double(h), ctypes.c_double(rtol),
                                    ctypes.c_double(atol), METHODS[method])

    def error_norm(self, q0, v0, q1, v1, e, rtol=1e-6, atol=1e-8):
        """The controller's error norm of an embedded difference e (2 nv tangent
        components) between the states (q0, v0) and (q1, v1)."""
        return lib().orc_error_norm(self.h, _p(_f64(q0)), _p(_f64(v0)), _p(_f64(q1)), _p(_f64(v1)), _p(_f64(e)),
                                    ctypes.c_double(rtol), ctypes.c_double(atol))

    def step_jacobian(self, q, v, u, h, cfd=False, method="dopri5"):
        Jx = np.zeros((self.nx, self.nx)); Ju = np.zeros((self.nx, max(self.nu, 1)))
        u = _f64(u if u is not None else np.zeros(max(self.nu, 1)))
        lib().orc_step_jacobian(self.h, _p(_f64(q)), _p(_f64(v)), _p(u), ctypes.c_double(h), int(cfd), _p(Jx), _p(Ju),
                                METHODS[method])
        return Jx, Ju[:, :self.nu]

    # ---------------------------------------------------------------- rollouts (one env)
    def rollout(self, x0, ctrl=None, T=1.0, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000, hcap=200000,
                method="dopri5"):
        xT = np.zeros(self.nx); xb = np.zeros((NI + 1, self.nx)); st = np.zeros(4, dtype=np.int32)
        hlog = np.zeros(hcap)
        c = _f64(ctrl) if ctrl is not None else _f64(np.zeros(max(NI * self.nu, 1)))
        n = lib().orc_rollout(self.h, _p(_f64(x0)), _p(c), ctypes.c_double(T), NI, ctypes.c_double(rtol),
                              ctypes.c_double(atol), ctypes.c_double(h0), max_steps, _p(xT), _p(xb), _p(st), _p(hlog), hcap,
                              METHODS[method])
        return {"xT": xT, "xb": xb, "status": int(st[0]), "nsteps": int(st[1]), "nrej": int(st[2]),
                "nrhs": int(st[3]), "hlog": hlog[:min(n, hcap)].copy()}

    def replay(self, x0, hlog, ctrl=None, T=1.0, NI=1, method="dopri5"):
        xT = np.zeros(self.nx); xb = np.zeros((NI + 1, self.nx))
        c = _f64(ctrl) if ctrl is not None else _f64(np.zeros(max(NI * self.nu, 1)))
        hl = _f64(hlog)
        lib().orc_replay(self.h, _p(_f64(x0)), _p(c), ctypes.c_double(T), NI, _p(hl), len(hl), _p(xT), _p(xb),
                         METHODS[method])
        return xT, xb

    def rollout_grad(self, x0, xT_bar, ctrl=None, T=1.0, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000,
                     cfd=False, xb_bar=None, method="dopri5"):
        xT = np.zeros(self.nx); gx = np.zeros(self.nx); gu = np.zeros(max(NI * self.nu, 1)); st = np.zeros(4, dtype=np.int32)
        c = _f64(ctrl) if ctrl is not None else _f64(np.zeros(max(NI * self.nu, 1)))
        xbb = _f64(xb_bar) if xb_bar is not None else None
        lib().orc_rollout_grad(self.h, _p(_f64(x0)), _p(c), ctypes.c_double(T), NI, ctypes.c_double(rtol),
                               ctypes.c_double(atol), ctypes.c_double(h0), max_steps, int(cfd), _p(_f64(xT_bar)),
                               _p(xbb), _p(xT), _p(gx), _p(gu), _p(st), METHODS[method])
        return {"xT": xT, "x0_bar": gx, "ctrl_bar": gu[:NI * self.nu].reshape(NI, self.nu), "status": int(st[0]),
                "nsteps": int(st[1])}

    def count_flops(self, x0, ctrl=None, T=1.0, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000, search=True,
                    method="dopri5"):
        """FP64 operations of one adaptive rollout (counting scalar).  search=False
        counts each constraint solve as started at its final active set (one
        Newton system plus one residual check) instead of the oracle's search
        from the unconstrained acceleration."""
        st = np.zeros(4, dtype=np.int32)
        c = _f64(ctrl) if ctrl is not None else _f64(np.zeros(max(NI * self.nu, 1)))
        n = lib().orc_count_flops(self.h, _p(_f64(x0)), _p(c), ctypes.c_double(T), NI, ctypes.c_double(rtol),
                                  ctypes.c_double(atol), ctypes.c_double(h0), max_steps, _p(st), int(bool(search)),
                                  METHODS[method])
        return int(n), {"status": int(st[0]), "nsteps": int(st[1]), "nrej": int(st[2]), "nrhs": int(st[3])}

    def count_adjoint_flops(self, x0, ctrl=None, T=1.0, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000,
                            method="dopri5"):
        """FP64 operations of the discrete adjoint of one rollout: every accepted
        step evaluated once with one tangent (primal recompute + linearised step)."""
        st = np.zeros(4, dtype=np.int32)
        c = _f64(ctrl) if ctrl is not None else _f64(np.zeros(max(NI * self.nu, 1)))
        n = lib().orc_count_adjoint_flops(self.h, _p(_f64(x0)), _p(c), ctypes.c_double(T), NI, ctypes.c_double(rtol),
                                          ctypes.c_double(atol), ctypes.c_double(h0), max_steps, _p(st),
                                          METHODS[method])
        return int(n), {"status": int(st[0]), "nsteps": int(st[1]), "nrej": int(st[2]), "nrhs": int(st[3])}

    # ---------------------------------------------------------------- batched (env-major arrays)
    def batch_rollout(self, x0, T, ctrl=None, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000, nthreads=None,
                      want_xb=False, method="dopri5"):
        x0 = _f64(x0)
        B = x0.shape[0]
        xT = np.zeros((B, self.nx)); st = np.zeros((B, 4), dtype=np.int32)
        xb = np.zeros((B, NI + 1, self.nx)) if want_xb else None
        c = _f64(ctrl) if (ctrl is not None and self.nu) else None
        lib().orc_batch_rollout(self.h, B, _p(x0), _p(c), _p(_f64(np.broadcast_to(T, (B,)))), NI,
                                ctypes.c_double(rtol), ctypes.c_double(atol), ctypes.c_double(h0), max_steps,
                                _p(xT), _p(xb), _p(st), int(nthreads or os.cpu_count() or 1), METHODS[method])
        return {"xT": xT, "xb": xb, "status": st[:, 0].copy(), "nsteps": st[:, 1].copy(), "nrej": st[:, 2].copy(),
                "nrhs": st[:, 3].copy()}

    def batch_replay_grad(self, x0, T, hlog, n, xT_bar, ctrl=None, NI=1, cfd=False, xb_bar=None, nthreads=None,
                          method="dopri5", params=False):
        """Discrete adjoint along given accepted step sizes (hlog [B, >= max n], n [B]);
        params=True adds "p_bar" [B, np]: the gradient w.r.t. the model parameters
        (solref t_c, phi_d; solimp d_o, d_w, width, midpoint; friction of each pair)."""
        x0 = _f64(x0)
        B = x0.shape[0]
        hlog = _f64(hlog)
        n = np.ascontiguousarray(np.asarray(n, dtype=np.int32))
        xT = np.zeros((B, self.nx)); gx = np.zeros((B, self.nx))
        gu = np.zeros((B, NI, self.nu)) if self.nu else None
        c = _f64(ctrl) if (ctrl is not None and self.nu) else None
        pb = np.zeros((B, self.nparams())) if params else None
        lib().orc_batch_replay_grad(self.h, B, _p(x0), _p(c), _p(_f64(np.broadcast_to(T, (B,)))), NI, _p(hlog),
                                    hlog.shape[1], _p(n), int(cfd), _p(_f64(xT_bar)),
                                    _p(_f64(xb_bar) if xb_bar is not None else None), _p(xT), _p(gx), _p(gu),
                                    int(nthreads or os.cpu_count() or 1), METHODS[method], _p(pb))
        out = {"xT": xT, "x0_bar": gx, "ctrl_bar": gu}
        if params:
            out["p_bar"] = pb
        return out

    def batch_grad_otd(self, x0, T, xT_bar, ctrl=None, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000,
                       cfd=False, xb_bar=None, nthreads=None, method="dopri5"):
        """Optimize-then-discretize (backsolve) gradient: the continuous adjoint
        integrated backward with the state, its own adaptive steps."""
        x0 = _f64(x0)
        B = x0.shape[0]
        xT = np.zeros((B, self.nx)); gx = np.zeros((B, self.nx)); st = np.zeros((B, 8), dtype=np.int32)
        gu = np.zeros((B, NI, self.nu)) if self.nu else None
        c = _f64(ctrl) if (ctrl is not None and self.nu) else None
        lib().orc_batch_grad_otd(self.h, B, _p(x0), _p(c), _p(_f64(np.broadcast_to(T, (B,)))), NI,
                                 ctypes.c_double(rtol), ctypes.c_double(atol), ctypes.c_double(h0), max_steps, int(cfd),
                                 _p(_f64(xT_bar)), _p(_f64(xb_bar) if xb_bar is not None else None), _p(xT), _p(gx),
                                 _p(gu), _p(st), int(nthreads or os.cpu_count() or 1), METHODS[method])
        return {"xT": xT, "x0_bar": gx, "ctrl_bar": gu, "status": st[:, 0].copy(), "nsteps": st[:, 1].copy(),
                "back_status": st[:, 4].copy(), "back_steps": st[:, 5].copy(), "back_rej": st[:, 6].copy()}

    def nparams(self):
        """Model parameters of the adjoint: t_c, phi_d, d_o, d_w, width, midpoint, mu of each pair,
        the mass of each body (its rotational inertia scaled in proportion), then the side length of
        each box geom (half sizes scaled together; the inertia of a body that is the box by the square)."""
        return int(lib().orc_nparams(self.h))

    def batch_grad(self, x0, T, xT_bar, ctrl=None, NI=1, rtol=1e-6, atol=1e-8, h0=1e-3, max_steps=20000, cfd=False,
                   xb_bar=None, nthreads=None, method="dopri5"):
        x0 = _f64(x0)
        B = x0.shape[0]
        xT = np.zeros((B, self.nx)); gx = np.zeros((B, self.nx)); st = np.zeros((B, 4), dtype=np.int32)
        gu = np.zeros((B, NI, self.nu)) if self.nu else None
        c = _f64(ctrl) if (ctrl is not None and self.nu) else None
        lib().orc_batch_grad(self.h, B, _p(x0), _p(c), _p(_f64(np.broadcast_to(T, (B,)))), NI,
                             ctypes.c_double(rtol), ctypes.c_double(atol), ctypes.c_double(h0), max_steps, int(cfd),
                             _p(_f64(xT_bar)), _p(_f64(xb_bar) if xb_bar is not None else None), _p(xT), _p(gx),
                             _p(gu), _p(st), int(nthreads or os.cpu_count() or 1), METHODS[method])
        return {"xT": xT, "x0_bar": gx, "ctrl_bar": gu, "status": st[:, 0].copy(), "nsteps": st[:, 1].copy()}


def tableau(method="dopri5"):
    """Coefficients the oracle integrates with: (a 7x7, b, bhat, c) of the
    explicit scheme (position coefficients equal to the velocity ones), or
    with partitioned=True style access through tableau_full."""
    t = tableau_full(method)
    return t["av"], t["b"], t["bhat"], t["c"]


def tableau_full(method="dopri5"):
    """All coefficients of a scheme: stages S, aq and av (7x7), b, bhat, c."""
    aq = np.zeros(49); av = np.zeros(49); b = np.zeros(7); bh = np.zeros(7); c = np.zeros(7)
    S = lib().orc_tableau(METHODS[method], _p(aq), _p(av), _p(b), _p(bh), _p(c))
    return {"S": int(S), "aq": aq.reshape(7, 7), "av": av.reshape(7, 7), "b": b, "bhat": bh, "c": c}
