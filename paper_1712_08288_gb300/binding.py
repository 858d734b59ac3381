"""Thin ctypes binding of liblbm.so (include/lbm.h).  Argument marshalling only:
every step of the computation runs in the library's CUDA kernels.

The library must have been built (``python -m paper_1712_08288_gb300._build`` or
``__graft_entry__.build()``); importing this module without it raises ImportError
-- there is no CPU fallback.
"""

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

LBM_D2Q9, LBM_D3Q19, LBM_D3Q15 = 0, 1, 2
LBM_F64, LBM_F32_DEV, LBM_BF16_DEV, LBM_F16_DEV = 0, 1, 2, 3
PRECISIONS = {"f64": LBM_F64, "f32": LBM_F32_DEV, "bf16": LBM_BF16_DEV, "f16": LBM_F16_DEV}
LATTICES = {"D2Q9": LBM_D2Q9, "D3Q19": LBM_D3Q19, "D3Q15": LBM_D3Q15}
STATUS = {0: "LBM_OK", -1: "LBM_EINVAL", -2: "LBM_ENOMEM", -3: "LBM_ECUDA",
          -4: "LBM_ENONCONVEX", -5: "LBM_EDIVERGED", -6: "LBM_ETIMEOUT", -7: "LBM_ESTATE"}

# every symbol include/lbm.h declares
EXPORTS = ["lbm_create", "lbm_destroy", "lbm_set_stream", "lbm_set_skew", "lbm_set_geometry",
           "lbm_set_scheme", "lbm_set_force", "lbm_set_wall_factor", "lbm_set_two_node", "lbm_init_equilibrium", "lbm_set_populations",
           "lbm_get_populations", "lbm_step", "lbm_time", "lbm_moments", "lbm_moments_device",
           "lbm_error_norms", "lbm_error_norms_noalloc", "lbm_query", "lbm_last_error",
           "lbm_set_relaxation", "lbm_set_link_values", "lbm_set_wait_limit", "lbm_adjoint",
           "lbm_adjoint_forward", "lbm_adjoint_backward", "lbm_probe_fp64_rate",
           "lbm_batch_create", "lbm_batch_destroy", "lbm_batch_set_stream", "lbm_batch_set_config",
           "lbm_batch_tune", "lbm_batch_step", "lbm_batch_query", "lbm_batch_last_error"]


class lbm_norms(ct.Structure):
    _fields_ = [("l2_rel", ct.c_double), ("linf", ct.c_double), ("mass", ct.c_double),
                ("mom", ct.c_double * 3), ("residual", ct.c_double)]


def load_library(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError("liblbm.so is not built (%s); run __graft_entry__.build()" % path)
    lib = ct.CDLL(path)
    P, D, I, I64 = ct.c_void_p, ct.c_double, ct.c_int, ct.c_int64
    sig = {
        "lbm_create": (I, [ct.POINTER(P), I, I, I, I, P, I, D]),
        "lbm_destroy": (I, [P]),
        "lbm_set_stream": (I, [P, P]),
        "lbm_set_skew": (I, [P, I, I]),
        "lbm_set_geometry": (I, [P, P, I64, P, P, P, P]),
        "lbm_set_scheme": (I, [P, D, D, D, D, I]),
        "lbm_set_force": (I, [P, P]),
        "lbm_set_wall_factor": (I, [P, D, D]),
        "lbm_set_two_node": (I, [P, I]),
        "lbm_init_equilibrium": (I, [P, P, P]),
        "lbm_set_populations": (I, [P, P]),
        "lbm_get_populations": (I, [P, P]),
        "lbm_step": (I, [P, I]),
        "lbm_time": (I64, [P]),
        "lbm_moments": (I, [P, P, P]),
        "lbm_moments_device": (I, [P, P, P]),
        "lbm_error_norms": (I, [P, P, ct.POINTER(lbm_norms)]),
        "lbm_error_norms_noalloc": (I, [P, P, P]),
        "lbm_query": (I, [P, P, P, P, P, P]),
        "lbm_last_error": (ct.c_char_p, [P]),
        "lbm_set_relaxation": (I, [P, P]),
        "lbm_set_link_values": (I, [P, P, P]),
        "lbm_set_wait_limit": (I, [P, I]),
        "lbm_adjoint": (I, [P, I, I, P, P, P, P, P, P]),
        "lbm_adjoint_forward": (I, [P, I, I, P, P, P]),
        "lbm_adjoint_backward": (I, [P, P, P, P]),
        "lbm_probe_fp64_rate": (I, [P]),
        "lbm_batch_create": (I, [ct.POINTER(P), I, P]),
        "lbm_batch_destroy": (I, [P]),
        "lbm_batch_set_stream": (I, [P, P]),
        "lbm_batch_set_config": (I, [P, I, I, I, I]),
        "lbm_batch_tune": (I, [P, I, P, P, P, P]),
        "lbm_batch_step": (I, [P, I]),
        "lbm_batch_query": (I, [P, P, P, P, P, P, P]),
        "lbm_batch_last_error": (ct.c_char_p, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


class LbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


class Lbm:
    """One simulation context (lbm_ctx).  Method names follow the C-ABI."""

    def __init__(self, lattice, shape, s, precision="f64", rho0=1.0):
        self._lib = lib()
        self.lattice = lattice
        self.lat_id = LATTICES[lattice]
        self.shape = tuple(int(v) for v in shape)
        self.precision = precision
        self.rho0 = float(rho0)
        self.Q = {"D2Q9": 9, "D3Q19": 19, "D3Q15": 15}[lattice]
        self.D = 2 if lattice == "D2Q9" else 3
        self.N = self.shape[0] * self.shape[1] * self.shape[2]
        s = np.ascontiguousarray(s, dtype=np.float64)
        assert s.shape == (self.Q,)
        h = ct.c_void_p()
        rc = self._lib.lbm_create(ct.byref(h), self.lat_id, *self.shape, _ptr(s),
                                  PRECISIONS[precision], self.rho0)
        if rc != 0:
            raise LbmError(rc, self._lib.lbm_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != 0:
            raise LbmError(rc, self._lib.lbm_last_error(self.h).decode())
        return rc

    def close(self):
        if getattr(self, "h", None):
            self._lib.lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- setup -------------------------------------------------------------
    def set_stream(self, stream_handle):
        self._check(self._lib.lbm_set_stream(self.h, ct.c_void_p(stream_handle)))

    def set_skew(self, sy, sz):
        self._check(self._lib.lbm_set_skew(self.h, int(sy), int(sz)))

    def set_geometry(self, solid, links):
        solid = np.ascontiguousarray(np.asarray(solid).reshape(self.N), dtype=np.uint8)
        node = np.ascontiguousarray(links["node"], dtype=np.int64)
        d = np.ascontiguousarray(links["d"], dtype=np.int32)
        q = np.ascontiguousarray(links["q"], dtype=np.float64)
        uw = links.get("uw")
        uw = None if uw is None else np.ascontiguousarray(np.asarray(uw, dtype=np.float64).reshape(-1, 3))
        self._check(self._lib.lbm_set_geometry(self.h, _ptr(solid), len(node), _ptr(node), _ptr(d),
                                               _ptr(q), _ptr(uw)))

    def set_scheme(self, c0, c1, c2, b=1.0, allow_nonconvex=False):
        self._check(self._lib.lbm_set_scheme(self.h, c0, c1, c2, b, int(bool(allow_nonconvex))))

    def set_force(self, g):
        g = np.ascontiguousarray(list(g) + [0.0] * (3 - len(g)), dtype=np.float64)
        self._check(self._lib.lbm_set_force(self.h, _ptr(g)))

    def set_two_node(self, enable=True):
        """lbm_set_two_node: Eq. 2.11 on the links whose x_l is fluid."""
        self._check(self._lib.lbm_set_two_node(self.h, int(bool(enable))))

    def set_wall_factor(self, a0=1.0, r=1.0):
        """lbm_set_wall_factor: wall velocities times a0 r^(t - now) at step t."""
        self._check(self._lib.lbm_set_wall_factor(self.h, float(a0), float(r)))

    def init_equilibrium(self, rho=None, u=None):
        rho = None if rho is None else np.ascontiguousarray(np.asarray(rho).reshape(self.N), dtype=np.float64)
        if u is not None:
            u = np.ascontiguousarray(np.asarray(u, dtype=np.float64).reshape(self.N, -1)[:, : self.D])
        self._check(self._lib.lbm_init_equilibrium(self.h, _ptr(rho), _ptr(u)))

    def set_populations(self, f):
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(self.Q, self.N))
        self._check(self._lib.lbm_set_populations(self.h, _ptr(f)))

    # -- run / read ----------------------------------------------------------
    def step(self, n=1):
        self._check(self._lib.lbm_step(self.h, int(n)))

    def time(self):
        return int(self._lib.lbm_time(self.h))

    def get_populations(self):
        f = np.empty((self.Q, self.N), dtype=np.float64)
        self._check(self._lib.lbm_get_populations(self.h, _ptr(f)))
        return f

    def moments(self):
        rho = np.empty(self.N, dtype=np.float64)
        u = np.empty((self.N, self.D), dtype=np.float64)
        self._check(self._lib.lbm_moments(self.h, _ptr(rho), _ptr(u)))
        return rho, u

    def moments_device(self, rho_ptr, u_ptr):
        self._check(self._lib.lbm_moments_device(self.h, ct.c_void_p(rho_ptr), ct.c_void_p(u_ptr)))

    def error_norms(self, u_ref=None, check=True):
        out = lbm_norms()
        if u_ref is not None:
            u_ref = np.ascontiguousarray(np.asarray(u_ref, dtype=np.float64).reshape(self.N, -1)[:, : self.D])
        rc = self._lib.lbm_error_norms(self.h, _ptr(u_ref), ct.byref(out))
        if check:
            self._check(rc)
        return dict(l2_rel=out.l2_rel, linf=out.linf, mass=out.mass, mom=list(out.mom),
                    residual=out.residual, status=rc)

    def error_norms_noalloc(self, u_ref_dev_ptr, out_dev_ptr):
        """lbm_error_norms_noalloc: device pointers in, nothing allocated, asynchronous."""
        self._check(self._lib.lbm_error_norms_noalloc(self.h, ct.c_void_p(u_ref_dev_ptr),
                                                      ct.c_void_p(out_dev_ptr)))

    def set_wait_limit(self, polls):
        """lbm_set_wait_limit: barrier polls before a sweep gives up (default 1000)."""
        self._check(self._lib.lbm_set_wait_limit(self.h, int(polls)))

    def set_relaxation(self, s):
        s = np.ascontiguousarray(s, dtype=np.float64)
        assert s.shape == (self.Q,)
        self._check(self._lib.lbm_set_relaxation(self.h, _ptr(s)))

    def set_link_values(self, q=None, uw=None):
        q = None if q is None else np.ascontiguousarray(q, dtype=np.float64)
        uw = None if uw is None else np.ascontiguousarray(np.asarray(uw, dtype=np.float64).reshape(-1, 3))
        self._check(self._lib.lbm_set_link_values(self.h, _ptr(q), _ptr(uw)))

    def adjoint(self, n_steps, mask, u_target, checkpoint_every=0):
        """lbm_adjoint: (J, dJ/ds (Q,), dJ/dq (links,), dJ/dphi (links, 3))."""
        nl = self.query()["links"]
        mask = np.ascontiguousarray(np.asarray(mask).reshape(self.N), dtype=np.uint8)
        ut = np.ascontiguousarray(np.asarray(u_target, dtype=np.float64).reshape(self.N, -1)[:, : self.D])
        J = ct.c_double()
        gs = np.zeros(self.Q)
        gq = np.zeros(nl)
        gp = np.zeros((nl, 3))
        self._check(self._lib.lbm_adjoint(self.h, int(n_steps), int(checkpoint_every), _ptr(mask), _ptr(ut),
                                          ct.byref(J), _ptr(gs), _ptr(gq), _ptr(gp)))
        return J.value, gs, gq, gp

    def adjoint_forward(self, n_steps, mask, u_target, checkpoint_every=0):
        """lbm_adjoint_forward: the checkpointed run; returns J and keeps the tape."""
        mask = np.ascontiguousarray(np.asarray(mask).reshape(self.N), dtype=np.uint8)
        ut = np.ascontiguousarray(np.asarray(u_target, dtype=np.float64).reshape(self.N, -1)[:, : self.D])
        J = ct.c_double()
        self._check(self._lib.lbm_adjoint_forward(self.h, int(n_steps), int(checkpoint_every), _ptr(mask),
                                                  _ptr(ut), ct.byref(J)))
        return J.value

    def adjoint_backward(self):
        """lbm_adjoint_backward: (dJ/ds (Q,), dJ/dq (links,), dJ/dphi (links, 3)) from the tape."""
        nl = self.query()["links"]
        gs = np.zeros(self.Q)
        gq = np.zeros(nl)
        gp = np.zeros((nl, 3))
        self._check(self._lib.lbm_adjoint_backward(self.h, _ptr(gs), _ptr(gq), _ptr(gp)))
        return gs, gq, gp

    def query(self):
        Q, D = ct.c_int(), ct.c_int()
        n, nf, nl = ct.c_int64(), ct.c_int64(), ct.c_int64()
        self._check(self._lib.lbm_query(self.h, ct.byref(Q), ct.byref(D), ct.byref(n), ct.byref(nf),
                                        ct.byref(nl)))
        return dict(Q=Q.value, D=D.value, nodes=n.value, fluid_nodes=nf.value, links=nl.value)


def probe_fp64_rate():
    """lbm_probe_fp64_rate: the current device's FP64 FMA rate in GFLOP/s."""
    g = ct.c_double()
    rc = lib().lbm_probe_fp64_rate(ct.byref(g))
    if rc != 0:
        raise LbmError(rc, "lbm_probe_fp64_rate failed")
    return g.value


def adjoint_loss_function():
    """A torch.autograd.Function for J = sum_mask |u(T) - u_target|^2 after n_steps
    from a fixed initial state.  forward runs lbm_adjoint_forward (the checkpointed
    run: the cost of the n_steps plus the checkpoint copies) and returns J;
    backward runs lbm_adjoint_backward (recompute and adjoint sweep) and returns
    gJ * dJ/dq per link, gJ * dJ/ds and gJ * dJ/dphi on the inputs' devices and
    dtypes.

    apply(q, s, uw, sim, f0, n_steps, mask, u_target, checkpoint_every) with q
    (links,), s (Q,), uw (links, 3) tensors (any device; their values are copied to
    the context); f0 the initial full populations (Q, nodes) numpy array the run
    starts from.  The context holds one tape: stepping or changing it between
    forward and backward makes backward raise (LBM_ESTATE).  J is returned on q's
    device in float64.
    """
    import torch

    class AdjointLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, q, s, uw, sim, f0, n_steps, mask, u_target, checkpoint_every=0):
            sim.set_relaxation(s.detach().to("cpu", torch.float64).numpy())
            sim.set_link_values(q.detach().to("cpu", torch.float64).numpy(),
                                uw.detach().to("cpu", torch.float64).numpy())
            sim.set_populations(f0)
            J = sim.adjoint_forward(n_steps, mask, u_target, checkpoint_every)
            ctx.sim = sim
            ctx.like = (q, s, uw)
            return torch.tensor(J, dtype=torch.float64, device=q.device)

        @staticmethod
        def backward(ctx, gJ):
            gs, gq, gp = ctx.sim.adjoint_backward()
            q, s, uw = ctx.like
            g = gJ.detach().to("cpu", torch.float64)
            out = []
            for grad, like in ((gq, q), (gs, s), (gp, uw)):
                t = g * torch.from_numpy(grad.reshape(tuple(like.shape)))
                out.append(t.to(like.device, like.dtype))
            return (out[0], out[1], out[2], None, None, None, None, None, None)

    return AdjointLoss


class Batch:
    """lbm_batch: several contexts advanced by one persistent launch per step."""

    ORDERS = {0: "context-major", 1: "round-robin", 2: "largest-first"}

    def __init__(self, sims):
        self._lib = lib()
        self.sims = list(sims)          # keep the contexts alive while the batch exists
        arr = (ct.c_void_p * len(self.sims))(*[s.h.value for s in self.sims])
        h = ct.c_void_p()
        rc = self._lib.lbm_batch_create(ct.byref(h), len(self.sims), ct.cast(arr, ct.c_void_p))
        if rc != 0:
            raise LbmError(rc, self._lib.lbm_batch_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != 0:
            raise LbmError(rc, self._lib.lbm_batch_last_error(self.h).decode())

    def set_stream(self, stream_handle):
        self._check(self._lib.lbm_batch_set_stream(self.h, ct.c_void_p(stream_handle)))

    def set_config(self, order, blocks_per_sm=0, split=1, tile_w=64):
        self._check(self._lib.lbm_batch_set_config(self.h, int(order), int(blocks_per_sm), int(split),
                                                   int(tile_w)))

    def tune(self, trial_steps=20):
        """lbm_batch_tune: (order, blocks_per_sm, split, tile_w) of the fastest configuration."""
        o, b, sp, w = ct.c_int(), ct.c_int(), ct.c_int(), ct.c_int()
        self._check(self._lib.lbm_batch_tune(self.h, int(trial_steps), ct.byref(o), ct.byref(b), ct.byref(sp),
                                             ct.byref(w)))
        return o.value, b.value, sp.value, w.value

    def step(self, n=1):
        self._check(self._lib.lbm_batch_step(self.h, int(n)))

    def query(self):
        n, t, o, b, k, w = ct.c_int(), ct.c_int64(), ct.c_int(), ct.c_int(), ct.c_int(), ct.c_int()
        self._check(self._lib.lbm_batch_query(self.h, ct.byref(n), ct.byref(t), ct.byref(o), ct.byref(b),
                                              ct.byref(k), ct.byref(w)))
        return dict(contexts=n.value, tiles=t.value, order=o.value, blocks_per_sm=b.value,
                    launches_per_step=k.value, tile_w=w.value)

    def close(self):
        if getattr(self, "h", None):
            self._lib.lbm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def from_workload(w, precision="f64", scheme=(0.0, 1.0, 0.0, 1.0), allow_nonconvex=False):
    """Build a context from an input-generator dict (workloads module)."""
    sim = Lbm(w["lattice"], w["shape"], w["S"], precision, w.get("rho0", 1.0))
    if tuple(w.get("skew", (0, 0))) != (0, 0):
        sim.set_skew(*w["skew"])
    sim.set_scheme(*scheme, allow_nonconvex=True)   # geometry not yet set: no links to check
    sim.set_geometry(w["solid"], w["links"])
    sim.set_scheme(*scheme, allow_nonconvex=allow_nonconvex)
    sim.set_force(w.get("force", (0.0, 0.0, 0.0)))
    return sim
