"""Python binding of libtde.so (include/tde.h): argument marshalling only.

Every computation runs in the CUDA library; PyTorch provides device memory and
the stream.  The binding raises if the library is missing or a call fails --
there is no CPU path.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

MATH_RCP, MATH_SQRT_RATIO, MATH_RCP_SEED, MATH_RSQRT_SEED, MATH_RSQRT, MATH_INSIDE = range(6)
TDE_OK, TDE_EINVAL, TDE_ENOMEM, TDE_ECUDA, TDE_ERANGE, TDE_ENUMERIC, TDE_ETIMEOUT = range(7)
EOS_IDEAL, EOS_TABLE = 0, 1
RECON_PLM, RECON_PPM = 0, 1
BC_OUTFLOW, BC_PERIODIC = 0, 1
RIEMANN_HLLC, RIEMANN_HLLE = 0, 1
INVERT_BISECT, INVERT_SURROGATE, INVERT_BISECT_PLAIN = 0, 1, 2
LAT_SEQUENCE, LAT_PERSISTENT = 0, 1
REMAP_THERMAL, REMAP_TOTAL = 0, 1
GRAV_PERIODIC, GRAV_ISOLATED = 0, 1
STATUS = {0: "TDE_OK", 1: "TDE_EINVAL", 2: "TDE_ENOMEM", 3: "TDE_ECUDA", 4: "TDE_ERANGE",
          5: "TDE_ENUMERIC", 6: "TDE_ETIMEOUT"}


class TDEError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


class Params(C.Structure):
    _fields_ = [("eos", C.c_int), ("recon", C.c_int), ("dual", C.c_int), ("gamma", C.c_double),
                ("eta1", C.c_double), ("eta2", C.c_double), ("rho_floor", C.c_double),
                ("p_floor", C.c_double), ("u_floor", C.c_double), ("unit_rho", C.c_double),
                ("unit_e", C.c_double), ("eos_mode", C.c_int), ("riemann", C.c_int)]


class BHState(C.Structure):
    _fields_ = [("on", C.c_int), ("excise", C.c_int), ("GM", C.c_double), ("r_soft", C.c_double),
                ("r_exc", C.c_double), ("t0", C.c_double), ("x0", C.c_double * 3),
                ("v0", C.c_double * 3), ("a0", C.c_double * 3), ("frame_on", C.c_int),
                ("afr", C.c_double * 3)]


class GravParams(C.Structure):
    _fields_ = [("G", C.c_double), ("rho_min", C.c_double), ("tol", C.c_double), ("max_cycles", C.c_int),
                ("npre", C.c_int), ("npost", C.c_int), ("omega", C.c_double), ("warm", C.c_int),
                ("boundary", C.c_int), ("lmax", C.c_int), ("fmg", C.c_int)]


class BlockDesc(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("i0", "j0", "k0", "nx", "ny", "nz", "level")]


def _block_descs(layout):
    nb = layout.nb
    return (BlockDesc * nb)(*[BlockDesc(*map(int, b), layout.level(q)) for q, b in enumerate(layout.blocks)])


class GridDesc(C.Structure):
    _fields_ = [("N", C.c_int * 3), ("xmin", C.c_double * 3), ("dx", C.c_double * 3),
                ("bc", C.c_int * 3), ("ng", C.c_int)]


class TableView(C.Structure):
    _fields_ = [("n_rho", C.c_int), ("n_T", C.c_int), ("log10_rho_min", C.c_double),
                ("log10_rho_max", C.c_double), ("log10_T_min", C.c_double),
                ("log10_T_max", C.c_double), ("log10_e", C.c_void_p), ("log10_P", C.c_void_p),
                ("log10_cs2", C.c_void_p)]


class Counts(C.Structure):
    _fields_ = [(n, C.c_uint64) for n in ("rho_floor", "p_floor", "u_floor", "table_clamp",
                                          "excised", "dual_aux_used", "synced", "nonfinite",
                                          "surrogate_accepted")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


class TrainReport(C.Structure):
    _fields_ = [("loss_first", C.c_double), ("loss_last", C.c_double), ("epochs", C.c_int),
                ("samples", C.c_int), ("batches", C.c_int), ("ms", C.c_double)]


vp = C.c_void_p
dp = C.c_void_p   # device pointers travel as integers
_SIGS = {
    "tde_init": [C.POINTER(vp), C.c_int, vp],
    "tde_set_stream": [vp, vp],
    "tde_finalize": [vp],
    "tde_eos_load_table": [vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double,
                           C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                           C.POINTER(vp)],
    "tde_eos_destroy": [vp],
    "tde_eos_invert": [vp, C.c_int, C.c_int64, dp, dp, dp, dp, dp, C.POINTER(Counts)],
    "tde_eos_eval_rhoT": [vp, C.c_int64, dp, dp, dp, dp, dp],
    "tde_eos_surrogate_train": [vp, C.c_uint64, C.c_int, C.c_int, C.c_int, C.c_double,
                                C.POINTER(TrainReport)],
    "tde_eos_surrogate_reset": [vp],
    "tde_eos_surrogate_set_weights": [vp, C.POINTER(C.c_float), C.c_size_t],
    "tde_eos_surrogate_get_weights": [vp, C.POINTER(C.c_float), C.c_size_t],
    "tde_eos_surrogate_grad": [vp, C.c_int64, dp, dp, dp, dp],
    "tde_eos_surrogate_forward": [vp, C.c_int64, dp, dp],
    "tde_eos_surrogate_norm": [vp, C.POINTER(C.c_double)],
    "tde_mesh_create": [vp, C.c_int, C.POINTER(BlockDesc), C.POINTER(GridDesc), C.POINTER(Params),
                        vp, C.POINTER(vp)],
    "tde_mesh_destroy": [vp],
    "tde_mesh_info": [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int), C.POINTER(C.c_int64)],
    "tde_mesh_set_params": [vp, C.POINTER(Params)],
    "tde_mesh_bind_state": [vp, dp, dp],
    "tde_prim_to_cons": [vp, dp, dp],
    "tde_ghost_fill": [vp, dp, C.c_int],
    "tde_hydro_stage": [vp, C.c_int, C.c_int, dp, dp, dp, C.POINTER(BHState)],
    "tde_compute_dt": [vp, C.c_double, dp, C.POINTER(BHState), dp, dp],
    "tde_excise": [vp, C.c_int, dp, dp, C.POINTER(BHState)],
    "tde_dual_energy_sync": [vp, C.c_int, dp, C.c_double],
    "tde_mesh_set_time": [vp, C.c_double],
    "tde_mesh_get_time": [vp, C.POINTER(C.c_double)],
    "tde_step": [vp, C.c_double, C.c_double, C.POINTER(BHState), dp],
    "tde_counts_read": [vp, C.POINTER(Counts), C.c_int],
    "tde_mesh_check": [vp],
    "tde_eos_check": [vp],
    "tde_eos_inject_wait_expiry": [vp, C.c_int],
    "tde_mesh_inject_wait_expiry": [vp, C.c_int],
    "tde_mesh_inject_barrier_drop": [vp, C.c_int],
    "tde_mesh_set_lat_mode": [vp, C.c_int, C.POINTER(C.c_int)],
    "tde_profile": [vp, C.c_int],
    "tde_profile_read": [vp, C.POINTER(C.c_uint64), C.POINTER(C.c_double)],
    "tde_probe_fp64": [vp, C.POINTER(C.c_double)],
    "tde_math_selftest": [vp, C.c_int64, dp, dp, dp],
    "tde_math_probe": [vp, C.c_int, C.c_int64, dp, dp, dp],
    "tde_riemann_probe": [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int64, dp, dp, dp, dp],
    "tde_mesh_autotune": [vp, C.POINTER(BHState), C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_float)],
    "tde_frame_acceleration": [vp, C.POINTER(BHState), C.c_double, C.POINTER(C.c_double),
                               C.POINTER(C.c_double)],
    "tde_mesh_boost": [vp, C.POINTER(C.c_double), C.c_double],
    "tde_gravity_solve": [vp, C.POINTER(GravParams), C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "tde_gravity_enable": [vp, C.c_int],
    "tde_gravity_phi": [vp, dp],
    "tde_mesh_remap": [vp, dp, vp, dp, C.c_int, C.c_double, C.c_double],
    "tde_mesh_set_tiles": [vp, C.POINTER(C.c_int32)],
    "tde_mesh_get_tiles": [vp, C.POINTER(C.c_int32)],
    "tde_lat_assign": [vp, C.c_int, C.c_double, C.c_double, C.POINTER(BHState), C.POINTER(C.c_int32),
                       C.POINTER(C.c_int), C.POINTER(C.c_double)],
    "tde_lat_set_factors": [vp, C.POINTER(C.c_int32), C.c_double],
    "tde_lat_window": [vp, C.POINTER(BHState), C.c_int, C.POINTER(C.c_int64)],
    "tde_compute_dt_noalloc": [vp, C.c_int, C.POINTER(BlockDesc), C.POINTER(GridDesc),
                               C.POINTER(Params), C.POINTER(TableView), dp, C.c_double, dp,
                               C.POINTER(BHState), dp, dp],
}
KERNEL_KINDS = ("c2p", "dt", "ghost", "sweep_x", "sweep_y", "sweep_z", "sync", "excise", "scalar",
                "p2c", "eos", "probe", "lat_graph", "grav", "remap", "lat_level")
NKIND = 16

_lib = None


def lib():
    """Load libtde.so (building it first if it is absent and nvcc is available)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            _build.build()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtde.so is missing: run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = C.c_int
        L.tde_last_error.argtypes = [vp]
        L.tde_last_error.restype = C.c_char_p
        _lib = L
    return _lib


def exported_symbols():
    return sorted(list(_SIGS) + ["tde_last_error"])


def _ptr(t):
    """Device pointer of a CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    return t.data_ptr()


class Context:
    """tde_ctx bound to a torch CUDA device and stream."""

    def __init__(self, device=0, stream=None):
        import torch
        self.torch = torch
        self.device = device
        s = stream if stream is not None else torch.cuda.current_stream(device)
        self.stream = s
        h = vp()
        self._check(lib().tde_init(C.byref(h), device, s.cuda_stream), None)
        self.h = h

    def _check(self, code, h="self"):
        if code != TDE_OK:
            msg = lib().tde_last_error(self.h if h == "self" else None)
            raise TDEError(code, msg.decode() if msg else "")

    def check(self, code):
        self._check(code)

    def profile(self, enable=True):
        self.check(lib().tde_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{kind: (launches, device ms)} since the last tde_profile() call."""
        n = (C.c_uint64 * NKIND)()
        ms = (C.c_double * NKIND)()
        self.check(lib().tde_profile_read(self.h, n, ms))
        return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(KERNEL_KINDS)}

    def probe_fp64(self):
        f = C.c_double()
        self.check(lib().tde_probe_fp64(self.h, C.byref(f)))
        return f.value

    def math_probe(self, op, x, out, y=None):
        self.check(lib().tde_math_probe(self.h, op, x.numel(), _ptr(x), _ptr(y), _ptr(out)))

    def riemann_probe(self, solver, d, wl, wr, F, vf, eos_table=1, dual=1, gamma=5.0 / 3.0):
        """The sweeps' Riemann solver on face-state pairs wl, wr [n][8] (device)."""
        self.check(lib().tde_riemann_probe(self.h, solver, d, eos_table, dual, gamma, wl.shape[0], _ptr(wl),
                                           _ptr(wr), _ptr(F), _ptr(vf)))

    def close(self):
        if getattr(self, "h", None):
            lib().tde_finalize(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class EOS:
    """tde_eos: a (log10 rho, log10 T) table copied to the device."""

    def __init__(self, ctx, n_rho, n_T, lrho, lT, log10_e, log10_P, log10_cs2):
        self.ctx = ctx
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (log10_e, log10_P, log10_cs2)]
        h = vp()
        ptrs = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in arrs]
        ctx.check(lib().tde_eos_load_table(ctx.h, n_rho, n_T, lrho[0], lrho[1], lT[0], lT[1],
                                           *ptrs, C.byref(h)))
        self.h = h
        self.n_rho, self.n_T, self.lrho, self.lT = n_rho, n_T, tuple(lrho), tuple(lT)

    @classmethod
    def from_file(cls, ctx, path):
        d = np.load(path)
        return cls(ctx, int(d["n_rho"]), int(d["n_T"]), tuple(d["lrho"]), tuple(d["lT"]),
                   d["log10_e"], d["log10_P"], d["log10_cs2"])

    def invert(self, rho, e, T=None, P=None, cs2=None, mode=INVERT_BISECT, counts=False):
        c = Counts() if counts else None
        self.ctx.check(lib().tde_eos_invert(self.h, mode, rho.numel(), _ptr(rho), _ptr(e), _ptr(T),
                                            _ptr(P), _ptr(cs2), C.byref(c) if c else None))
        return c

    def counts(self):
        c = Counts()
        self.ctx.check(lib().tde_eos_invert(self.h, INVERT_BISECT, 0, None, None, None, None, None,
                                            C.byref(c)))
        return c.as_dict()

    def check(self):
        """Raise TDEError (TDE_ETIMEOUT) if a bounded wait of the learned-guess
        inference expired since the last check."""
        self.ctx.check(lib().tde_eos_check(self.h))

    def inject_wait_expiry(self, on=True):
        """Failure-detection test hook: the inference's bounded wait expires."""
        self.ctx.check(lib().tde_eos_inject_wait_expiry(self.h, 1 if on else 0))

    def set_weights(self, w):
        a = np.ascontiguousarray(w, dtype=np.float32)
        self.ctx.check(lib().tde_eos_surrogate_set_weights(self.h, a.ctypes.data_as(C.POINTER(C.c_float)),
                                                           a.size))

    def get_weights(self):
        a = np.zeros(4482, dtype=np.float32)
        self.ctx.check(lib().tde_eos_surrogate_get_weights(self.h, a.ctypes.data_as(C.POINTER(C.c_float)),
                                                           a.size))
        return a

    def reset_weights_for_training(self):
        self.ctx.check(lib().tde_eos_surrogate_reset(self.h))

    def train(self, seed=0, n_samples=1 << 20, epochs=20, batch=8192, lr=3e-3):
        r = TrainReport()
        self.ctx.check(lib().tde_eos_surrogate_train(self.h, seed, n_samples, epochs, batch, lr,
                                                     C.byref(r)))
        return {n: getattr(r, n) for n, _ in r._fields_}

    def grad(self, x, target, grad, loss):
        self.ctx.check(lib().tde_eos_surrogate_grad(self.h, x.shape[0], _ptr(x), _ptr(target),
                                                    _ptr(grad), _ptr(loss)))

    def forward(self, x, y):
        self.ctx.check(lib().tde_eos_surrogate_forward(self.h, x.shape[0], _ptr(x), _ptr(y)))

    def math_selftest(self, x, log10_out=None, exp10_out=None):
        self.ctx.check(lib().tde_math_selftest(self.h, x.numel(), _ptr(x), _ptr(log10_out),
                                               _ptr(exp10_out)))

    def norm(self):
        out = (C.c_double * 8)()
        self.ctx.check(lib().tde_eos_surrogate_norm(self.h, out))
        return list(out)

    def eval_rhoT(self, rho, T, P=None, e=None, cs2=None):
        self.ctx.check(lib().tde_eos_eval_rhoT(self.h, rho.numel(), _ptr(rho), _ptr(T), _ptr(P),
                                               _ptr(e), _ptr(cs2)))

    def close(self):
        if getattr(self, "h", None):
            lib().tde_eos_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_params(**kw):
    p = Params(EOS_IDEAL, RECON_PLM, 0, 5.0 / 3.0, 1e-3, 1e-4, 1e-300, 1e-300, 1e-300, 1.0, 1.0, 0, 0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def make_bh(on=1, excise=0, GM=0.0, r_soft=0.0, r_exc=0.0, t0=0.0, x0=(0, 0, 0), v0=(0, 0, 0),
            a0=(0, 0, 0), frame_on=0, afr=(0, 0, 0)):
    return BHState(on, excise, GM, r_soft, r_exc, t0, (C.c_double * 3)(*x0),
                   (C.c_double * 3)(*v0), (C.c_double * 3)(*a0), frame_on, (C.c_double * 3)(*afr))


class Mesh:
    """tde_mesh over a workloads.MeshLayout, with torch-owned states U and U1."""

    def __init__(self, ctx, layout, params, eos=None):
        torch = ctx.torch
        self.ctx, self.layout, self.params, self.eos = ctx, layout, params, eos
        nb = layout.nb
        blocks = _block_descs(layout)
        g = GridDesc((C.c_int * 3)(*layout.N), (C.c_double * 3)(*layout.xmin),
                     (C.c_double * 3)(*layout.dx), (C.c_int * 3)(*layout.bc), layout.ng)
        h = vp()
        ctx.check(lib().tde_mesh_create(ctx.h, nb, blocks, C.byref(g), C.byref(params),
                                        eos.h if eos is not None else None, C.byref(h)))
        self.h = h
        ntot, nvar = C.c_int64(), C.c_int()
        offs = (C.c_int64 * (nb + 1))()
        ctx.check(lib().tde_mesh_info(h, C.byref(ntot), C.byref(nvar), offs))
        self.ntot, self.nvar = ntot.value, nvar.value
        self.offsets = np.array(offs[:], dtype=np.int64)
        dev = torch.device("cuda", ctx.device)
        self.U = torch.zeros((self.nvar, self.ntot), dtype=torch.float64, device=dev)
        self.U1 = torch.zeros_like(self.U)
        ctx.check(lib().tde_mesh_bind_state(h, _ptr(self.U), _ptr(self.U1)))

    def set_params(self, params):
        self.ctx.check(lib().tde_mesh_set_params(self.h, C.byref(params)))
        self.params = params

    def bind(self, U, U1=None):
        """Bind other caller-owned device states (nvar x ntot each) as U (and U1)."""
        self.U = U
        if U1 is not None:
            self.U1 = U1
        self.ctx.check(lib().tde_mesh_bind_state(self.h, _ptr(self.U), _ptr(self.U1)))

    def prim_to_cons(self, W):
        self.ctx.check(lib().tde_prim_to_cons(self.h, _ptr(W), _ptr(self.U)))

    def ghost_fill(self, state, nvar=None):
        self.ctx.check(lib().tde_ghost_fill(self.h, _ptr(state), nvar or self.nvar))

    def hydro_stage(self, stage, dt_block, t_block=None, ids=None, bh=None):
        n = 0 if ids is None else ids.numel()
        self.ctx.check(lib().tde_hydro_stage(self.h, stage, n, _ptr(ids), _ptr(dt_block),
                                             _ptr(t_block), C.byref(bh) if bh is not None else None))

    def compute_dt(self, cfl, dt_block, dt_min=None, t_block=None, bh=None):
        self.ctx.check(lib().tde_compute_dt(self.h, cfl, _ptr(t_block),
                                            C.byref(bh) if bh is not None else None,
                                            _ptr(dt_block), _ptr(dt_min)))

    def excise(self, t_end_block, bh, ids=None):
        n = 0 if ids is None else ids.numel()
        self.ctx.check(lib().tde_excise(self.h, n, _ptr(ids), _ptr(t_end_block), C.byref(bh)))

    def dual_energy_sync(self, ids=None, eta2=-1.0):
        n = 0 if ids is None else ids.numel()
        self.ctx.check(lib().tde_dual_energy_sync(self.h, n, _ptr(ids), eta2))

    def set_time(self, t):
        self.ctx.check(lib().tde_mesh_set_time(self.h, t))

    def get_time(self):
        t = C.c_double()
        self.ctx.check(lib().tde_mesh_get_time(self.h, C.byref(t)))
        return t.value

    def step(self, cfl=0.0, dt=0.0, bh=None, dt_out=None):
        self.ctx.check(lib().tde_step(self.h, cfl, dt, C.byref(bh) if bh is not None else None,
                                      _ptr(dt_out)))

    def lat_assign(self, n_lat, cfl, merge_frac=0.01, bh=None):
        f = (C.c_int32 * self.layout.nb)()
        fmax, dt0 = C.c_int(), C.c_double()
        self.ctx.check(lib().tde_lat_assign(self.h, n_lat, merge_frac, cfl,
                                            C.byref(bh) if bh is not None else None, f,
                                            C.byref(fmax), C.byref(dt0)))
        return np.array(f[:], dtype=np.int32), dt0.value, fmax.value

    def lat_set_factors(self, factors, dt0):
        f = np.ascontiguousarray(factors, dtype=np.int32)
        self.ctx.check(lib().tde_lat_set_factors(self.h, f.ctypes.data_as(C.POINTER(C.c_int32)), dt0))

    def lat_window(self, bh=None, use_graph=False):
        upd = C.c_int64()
        self.ctx.check(lib().tde_lat_window(self.h, C.byref(bh) if bh is not None else None,
                                            1 if use_graph else 0, C.byref(upd)))
        return upd.value

    def frame_acceleration(self, bh, rho_min):
        """(A_fr[3], mass) of Eq. frame-acceleration at the mesh time."""
        A = (C.c_double * 3)()
        mass = C.c_double()
        self.ctx.check(lib().tde_frame_acceleration(self.h, C.byref(bh), rho_min, A, C.byref(mass)))
        return list(A), mass.value

    def gravity_solve(self, G, rho_min, tol=1e-10, max_cycles=20, npre=2, npost=2, omega=1.15, warm=True,
                      isolated=False, lmax=4, fmg=False):
        """Self-gravity potential from the bound state's density; returns (cycles, rms defect)."""
        gp = GravParams(G, rho_min, tol, max_cycles, npre, npost, omega, 1 if warm else 0,
                        GRAV_ISOLATED if isolated else GRAV_PERIODIC, lmax, 1 if fmg else 0)
        n, d = C.c_int(), C.c_double()
        self.ctx.check(lib().tde_gravity_solve(self.h, C.byref(gp), C.byref(n), C.byref(d)))
        return n.value, d.value

    def gravity_enable(self, on=True):
        self.ctx.check(lib().tde_gravity_enable(self.h, 1 if on else 0))

    def gravity_phi(self):
        """The potential on the global grid, [Nz, Ny, Nx] (a CUDA tensor)."""
        import torch
        N = self.layout.N
        out = torch.empty((N[2], N[1], N[0]), dtype=torch.float64, device=self.U.device)
        self.ctx.check(lib().tde_gravity_phi(self.h, _ptr(out)))
        return out

    def remap_from(self, src, Usrc, mode=REMAP_THERMAL, rho_floor=None, u_floor=None, out=None):
        """Sec. 5.2 remap of src's state Usrc onto this mesh's interior cells (into
        out, default this mesh's U); the floors default to this mesh's."""
        out = self.U if out is None else out
        rf = self.params.rho_floor if rho_floor is None else rho_floor
        uf = self.params.u_floor if u_floor is None else u_floor
        self.ctx.check(lib().tde_mesh_remap(self.h, _ptr(out), src.h, _ptr(Usrc), mode, rf, uf))
        return out

    def boost(self, V, rho_min):
        v = (C.c_double * 3)(*V)
        self.ctx.check(lib().tde_mesh_boost(self.h, v, rho_min))

    def autotune(self, bh=None, reps=3):
        """Pick the fastest sweep tile shape per direction; returns (shapes, ms[3][3])."""
        t = (C.c_int32 * 3)()
        ms = (C.c_float * 9)()
        self.ctx.check(lib().tde_mesh_autotune(self.h, C.byref(bh) if bh is not None else None, reps,
                                               t, ms))
        return list(t), [list(ms[3 * d:3 * d + 3]) for d in range(3)]

    def set_tiles(self, tiles):
        t = (C.c_int32 * 3)(*tiles)
        self.ctx.check(lib().tde_mesh_set_tiles(self.h, t))

    def get_tiles(self):
        t = (C.c_int32 * 3)()
        self.ctx.check(lib().tde_mesh_get_tiles(self.h, t))
        return list(t)

    def inject_wait_expiry(self, on=True):
        """Failure-detection test hook: the sweeps' TMA waits expire (no copy issued)."""
        self.ctx.check(lib().tde_mesh_inject_wait_expiry(self.h, 1 if on else 0))

    def set_lat_mode(self, mode):
        """LAT_SEQUENCE or LAT_PERSISTENT (one cooperative launch per level
        sub-step); returns whether the mesh's current scheme takes the
        persistent form."""
        active = C.c_int(0)
        self.ctx.check(lib().tde_mesh_set_lat_mode(self.h, int(mode), C.byref(active)))
        return bool(active.value)

    def inject_barrier_drop(self, on=True):
        """Failure-detection test hook: the persistent level launch's first grid
        barrier is missing one arrival, so its bounded waits expire."""
        self.ctx.check(lib().tde_mesh_inject_barrier_drop(self.h, 1 if on else 0))

    def counts(self, reset=False):
        c = Counts()
        self.ctx.check(lib().tde_counts_read(self.h, C.byref(c), 1 if reset else 0))
        return c.as_dict()

    def check(self):
        """Raise TDEError (TDE_ENUMERIC: non-finite results counted since the last
        counter reset; TDE_ETIMEOUT: an expired wait of the sweeps' staging or of
        the learned guess)."""
        self.ctx.check(lib().tde_mesh_check(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib().tde_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def compute_dt_noalloc(ctx, layout, params, U, cfl, dt_block=None, dt_min=None, table=None,
                       t_block=None, bh=None):
    """tde_compute_dt_noalloc: per-block CFL step with no device allocation inside
    the library.  `table` is a (n_rho, n_T, lrho, lT, log10_e, log10_P, log10_cs2)
    tuple whose arrays are CUDA tensors the caller owns."""
    nb = layout.nb
    blocks = _block_descs(layout)
    g = GridDesc((C.c_int * 3)(*layout.N), (C.c_double * 3)(*layout.xmin),
                 (C.c_double * 3)(*layout.dx), (C.c_int * 3)(*layout.bc), layout.ng)
    tv = None
    if table is not None:
        n_rho, n_T, lrho, lT, le, lp, lc = table
        tv = TableView(n_rho, n_T, lrho[0], lrho[1], lT[0], lT[1], _ptr(le), _ptr(lp), _ptr(lc))
    ctx.check(lib().tde_compute_dt_noalloc(ctx.h, nb, blocks, C.byref(g), C.byref(params),
                                           C.byref(tv) if tv is not None else None, _ptr(U), cfl,
                                           _ptr(t_block), C.byref(bh) if bh is not None else None,
                                           _ptr(dt_block), _ptr(dt_min)))
