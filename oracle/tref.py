"""ctypes binding of the ORACLE (oracle/tref.h).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check in
__graft_entry__.py and by the CPU-baseline leg of bench.py.  Nothing in the
product package imports it.

The library is compiled from the C sources beside this file with
``-O2 -ffp-contract=off`` (every floating-point operation rounded as written)
and OpenMP over MeshBlocks.
"""
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libtref.so")
SOURCES = ["tref_eos.c", "tref_hydro.c", "tref_mlp.c", "tref_lat.c", "tref_grav.c", "tref_remap.c"]

EOS_IDEAL, EOS_TABLE = 0, 1
PLM, PPM = 0, 1
OUTFLOW, PERIODIC = 0, 1
HLLC, HLLE = 0, 1
REMAP_THERMAL, REMAP_TOTAL = 0, 1
MLP_NPARAM = 4482


def build(force=False):
    """Compile libtref.so (gcc, plain C11, no fp contraction)."""
    srcs = [os.path.join(HERE, s) for s in SOURCES if os.path.exists(os.path.join(HERE, s))]
    os.makedirs(BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(HERE, "tref.h")])
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= newest:
        return SO
    tmp = SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, SO)
    return SO


class Table(C.Structure):
    _fields_ = [("n_rho", C.c_int), ("n_T", C.c_int), ("lrho_min", C.c_double),
                ("lrho_max", C.c_double), ("lT_min", C.c_double), ("lT_max", C.c_double),
                ("log10_e", C.POINTER(C.c_double)), ("log10_P", C.POINTER(C.c_double)),
                ("log10_cs2", C.POINTER(C.c_double))]


class Params(C.Structure):
    _fields_ = [("eos", C.c_int), ("recon", C.c_int), ("dual", C.c_int), ("gamma", C.c_double),
                ("eta1", C.c_double), ("eta2", C.c_double), ("rho_floor", C.c_double),
                ("p_floor", C.c_double), ("u_floor", C.c_double), ("unit_rho", C.c_double),
                ("unit_e", C.c_double), ("bh_on", C.c_int), ("excision_on", C.c_int),
                ("GM", C.c_double), ("r_soft", C.c_double), ("r_exc", C.c_double),
                ("bh_t0", C.c_double), ("bh_x0", C.c_double * 3), ("bh_v0", C.c_double * 3),
                ("bh_a0", C.c_double * 3), ("riemann", C.c_int), ("frame_on", C.c_int),
                ("afr", C.c_double * 3)]


class MeshDesc(C.Structure):
    _fields_ = [("nb", C.c_int), ("blocks", C.POINTER(C.c_int)), ("N", C.c_int * 3),
                ("xmin", C.c_double * 3), ("dx", C.c_double * 3), ("bc", C.c_int * 3),
                ("ng", C.c_int), ("levels", C.POINTER(C.c_int))]


class Counts(C.Structure):
    _fields_ = [(n, C.c_int64) for n in
                ("rho_floor", "p_floor", "u_floor", "table_clamp", "excised", "dual_aux_used",
                 "synced")]

    def as_dict(self):
        return {n: int(getattr(self, n)) for n, _ in self._fields_}


_lib = None
dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int)
i32p = C.POINTER(C.c_int32)
i64p = C.POINTER(C.c_int64)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(SO)
        sig = {
            "tref_num_threads": (C.c_int, []),
            "tref_remap": (None, [C.c_void_p, dp, C.c_void_p, dp, C.c_int, C.c_double, C.c_double]),
            "tref_set_phi_sg": (None, [C.c_void_p, dp]),
            "tref_mg_solve": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_int, C.c_double,
                                        C.c_int, C.c_int, C.c_double, dp]),
            "tref_mg_defect_rms": (C.c_double, [C.c_int, C.c_int, C.c_int, dp, dp, dp]),
            "tref_mg_prolong": (None, [ip, ip, C.c_int, dp, dp]),
            "tref_mg_solve_bc": (C.c_int, [C.c_int, C.c_int, C.c_int, dp, dp, C.c_int, C.c_int, dp, C.c_int,
                                           dp, dp, C.c_int, C.c_double, C.c_int, C.c_int, C.c_double, dp, dp,
                                           C.c_int, dp, dp]),
            "tref_frame_acceleration": (None, [C.c_void_p, dp, C.c_double, C.c_double, dp, dp]),
            "tref_boost": (None, [C.c_void_p, dp, dp, C.c_double]),
            "tref_saha_state": (None, [C.c_double, C.c_double, C.c_double, C.c_double, dp]),
            "tref_saha_pure_h_xe": (C.c_double, [C.c_double, C.c_double]),
            "tref_eos_build": (None, [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_double, dp, dp, dp, dp]),
            "tref_eos_eval_rhoT": (None, [C.POINTER(Table), C.c_double, C.c_double, dp, dp, dp]),
            "tref_eos_eval_rhoT_n": (None, [C.POINTER(Table), C.c_int64, dp, dp, dp, dp, dp]),
            "tref_eos_invert": (C.c_int, [C.POINTER(Table), C.c_double, C.c_double, dp, dp, dp, dp]),
            "tref_eos_T_from_P": (C.c_double, [C.POINTER(Table), C.c_double, C.c_double]),
            "tref_eos_invert_guess": (C.c_int, [C.POINTER(Table), C.c_double, C.c_double, C.c_double,
                                                dp, dp, dp]),
            "tref_mesh_new": (C.c_void_p, [C.POINTER(MeshDesc), C.POINTER(Params), C.POINTER(Table)]),
            "tref_mesh_free": (None, [C.c_void_p]),
            "tref_mesh_ntot": (C.c_int64, [C.c_void_p]),
            "tref_mesh_block_offset": (C.c_int64, [C.c_void_p, C.c_int]),
            "tref_set_num_threads": (None, [C.c_int]),
            "tref_nvar": (C.c_int, [C.c_void_p]),
            "tref_set_params": (None, [C.c_void_p, C.POINTER(Params)]),
            "tref_ghost_fill": (None, [C.c_void_p, dp, C.c_int, C.c_int, ip]),
            "tref_ghost_fill_modes": (None, [C.c_void_p, dp, dp, dp, ip, dp, C.c_int, ip]),
            "tref_freg_block_size": (C.c_int64, [C.c_void_p, C.c_int]),
            "tref_cons_to_prim": (None, [C.c_void_p, dp, dp, C.POINTER(Counts)]),
            "tref_stage": (None, [C.c_void_p, C.c_int, C.c_int, ip, dp, dp, dp, dp, dp, dp,
                                  C.POINTER(Counts)]),
            "tref_excise": (None, [C.c_void_p, dp, C.c_int, ip, dp, C.POINTER(Counts)]),
            "tref_dual_sync": (None, [C.c_void_p, dp, C.c_int, ip, C.POINTER(Counts)]),
            "tref_cfl_dt": (None, [C.c_void_p, dp, C.c_double, dp, dp, C.POINTER(Counts)]),
            "tref_step": (None, [C.c_void_p, dp, dp, C.c_double, C.c_double, C.POINTER(Counts)]),
            "tref_prim_to_cons": (None, [C.c_void_p, dp, dp]),
            "tref_phi_bh": (C.c_double, [C.POINTER(Params), dp, C.c_double]),
            "tref_riemann": (None, [C.c_int, C.c_int, C.c_int, C.c_int64, dp, dp, dp, dp]),
            "tref_mlp_forward": (None, [dp, C.c_int64, dp, dp]),
            "tref_mlp_loss_grad": (C.c_double, [dp, C.c_int64, dp, dp, dp]),
        }
        optional = {
            "tref_lat_factors": (C.c_int, [C.c_void_p, dp, C.c_int, C.c_double, i32p, dp]),
            "tref_lat_window": (C.c_int, [C.c_void_p, dp, i32p, C.c_double, C.c_double,
                                          C.POINTER(Counts), i64p]),
        }
        for name, (res, args) in list(sig.items()) + list(optional.items()):
            if not hasattr(L, name):
                if name in optional:
                    continue
                raise AttributeError(name)
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def P(a):
    """numpy float64 array -> double*"""
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(dp)


def IP(a):
    assert a.dtype == np.int32 and a.flags.c_contiguous
    return a.ctypes.data_as(ip)


# ----------------------------------------------------------------- EOS ---

class EOSTable:
    """A (log10 rho, log10 T) table held in numpy arrays, with its ctypes view."""

    def __init__(self, n_rho, n_T, lrho, lT, log10_e, log10_P, log10_cs2, gamma1=None):
        self.n_rho, self.n_T, self.lrho, self.lT = n_rho, n_T, tuple(lrho), tuple(lT)
        self.log10_e = np.ascontiguousarray(log10_e, dtype=np.float64)
        self.log10_P = np.ascontiguousarray(log10_P, dtype=np.float64)
        self.log10_cs2 = np.ascontiguousarray(log10_cs2, dtype=np.float64)
        self.gamma1 = gamma1
        self.c = Table(n_rho, n_T, lrho[0], lrho[1], lT[0], lT[1], P(self.log10_e),
                       P(self.log10_P), P(self.log10_cs2))

    @classmethod
    def saha(cls, n_rho=256, n_T=256, lrho=(-14.0, 2.0), lT=(2.0, 8.0), X=0.7, Y=0.3):
        shape = (n_rho, n_T)
        le, lp, lc, g1 = (np.zeros(shape) for _ in range(4))
        lib().tref_eos_build(n_rho, n_T, lrho[0], lrho[1], lT[0], lT[1], X, Y, P(le), P(lp),
                             P(lc), P(g1))
        return cls(n_rho, n_T, lrho, lT, le, lp, lc, g1)

    def invert(self, rho, e):
        T, Pr, c2, eu = C.c_double(), C.c_double(), C.c_double(), C.c_double()
        cl = lib().tref_eos_invert(C.byref(self.c), rho, e, C.byref(T), C.byref(Pr), C.byref(c2),
                                   C.byref(eu))
        return T.value, Pr.value, c2.value, bool(cl)

    def eval_rhoT(self, rho, T):
        Pr, e, c2 = C.c_double(), C.c_double(), C.c_double()
        lib().tref_eos_eval_rhoT(C.byref(self.c), rho, T, C.byref(Pr), C.byref(e), C.byref(c2))
        return Pr.value, e.value, c2.value

    def eval_rhoT_n(self, rho, T):
        """(P, e, cs2) arrays at arrays (rho, T), cgs."""
        rho = np.ascontiguousarray(rho, dtype=np.float64).ravel()
        T = np.ascontiguousarray(T, dtype=np.float64).ravel()
        out = [np.empty_like(rho) for _ in range(3)]
        lib().tref_eos_eval_rhoT_n(C.byref(self.c), rho.size, P(rho), P(T), P(out[0]), P(out[1]), P(out[2]))
        return out

    def invert_guess(self, rho, e, log10_T_guess):
        T, Pr, c2 = C.c_double(), C.c_double(), C.c_double()
        acc = lib().tref_eos_invert_guess(C.byref(self.c), rho, e, log10_T_guess, C.byref(T),
                                          C.byref(Pr), C.byref(c2))
        return T.value, Pr.value, c2.value, bool(acc)

    def T_from_P(self, rho, Pr):
        return lib().tref_eos_T_from_P(C.byref(self.c), rho, Pr)


def saha_state(rho, T, X=0.7, Y=0.3):
    out = np.zeros(9)
    lib().tref_saha_state(rho, T, X, Y, P(out))
    keys = ("P", "e", "ne", "xH", "yHe1", "yHe2", "mu", "Pgas", "nnuc")
    return dict(zip(keys, out))


# ---------------------------------------------------------------- mesh ---

def make_params(**kw):
    p = Params()
    p.eos, p.recon, p.dual, p.gamma = EOS_IDEAL, PLM, 0, 5.0 / 3.0
    p.eta1, p.eta2 = 1e-3, 1e-4
    p.rho_floor, p.p_floor, p.u_floor = 1e-300, 1e-300, 1e-300
    p.unit_rho, p.unit_e = 1.0, 1.0
    p.bh_on = p.excision_on = 0
    p.GM = p.r_soft = p.r_exc = p.bh_t0 = 0.0
    p.riemann = HLLC
    for k, v in kw.items():
        if k in ("bh_x0", "bh_v0", "bh_a0", "afr"):
            setattr(p, k, (C.c_double * 3)(*v))
        else:
            setattr(p, k, v)
    return p


class Mesh:
    """Oracle mesh.  `layout` is a workloads.MeshLayout (blocks, N, xmin, dx, bc, ng)."""

    def __init__(self, layout, params, table=None):
        lib()
        self.layout = layout
        self.params = params
        self.table = table
        self._blocks = np.ascontiguousarray(layout.blocks, dtype=np.int32).reshape(-1)
        d = MeshDesc()
        d.nb = layout.nb
        d.blocks = self._blocks.ctypes.data_as(ip)
        d.N = (C.c_int * 3)(*layout.N)
        d.xmin = (C.c_double * 3)(*layout.xmin)
        d.dx = (C.c_double * 3)(*layout.dx)
        d.bc = (C.c_int * 3)(*layout.bc)
        d.ng = layout.ng
        lev = getattr(layout, "levels", None)
        self._levels = None if lev is None else np.ascontiguousarray(lev, dtype=np.int32)
        d.levels = self._levels.ctypes.data_as(ip) if self._levels is not None else None
        self.desc = d
        self.h = lib().tref_mesh_new(C.byref(d), C.byref(params),
                                     C.byref(table.c) if table is not None else None)
        if not self.h:
            raise ValueError("invalid mesh layout")
        self.ntot = lib().tref_mesh_ntot(self.h)
        self.nvar = lib().tref_nvar(self.h)

    def __del__(self):
        if getattr(self, "h", None):
            lib().tref_mesh_free(self.h)
            self.h = None

    def set_params(self, params):
        self.params = params
        lib().tref_set_params(self.h, C.byref(params))

    def new_state(self):
        return np.zeros((self.nvar, self.ntot))

    def prim_to_cons(self, W):
        U = self.new_state()
        lib().tref_prim_to_cons(self.h, P(np.ascontiguousarray(W)), P(U))
        return U

    def ghost_fill(self, U, nvar=None, ids=None):
        ids_a = None if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        lib().tref_ghost_fill(self.h, P(U), nvar or self.nvar, 0 if ids is None else len(ids_a),
                              None if ids_a is None else IP(ids_a))

    def stage(self, stage, U0, Uin, Uout, dt_b, t_b, ids=None, flux_reg=None, counts=None):
        ids_a = None if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        c = counts if counts is not None else Counts()
        lib().tref_stage(self.h, stage, 0 if ids_a is None else len(ids_a),
                         None if ids_a is None else IP(ids_a), P(U0), P(Uin), P(Uout),
                         P(np.ascontiguousarray(dt_b, dtype=np.float64)),
                         P(np.ascontiguousarray(t_b, dtype=np.float64)),
                         None if flux_reg is None else P(flux_reg), C.byref(c))
        return c

    def excise(self, U, t_end_b, ids=None, counts=None):
        ids_a = None if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        c = counts if counts is not None else Counts()
        lib().tref_excise(self.h, P(U), 0 if ids_a is None else len(ids_a),
                          None if ids_a is None else IP(ids_a),
                          P(np.ascontiguousarray(t_end_b, dtype=np.float64)), C.byref(c))
        return c

    def cons_to_prim(self, u, counts=None):
        """a2 + a3 on one cell: conserved u (5 or 6 values) -> primitives w[8]
        (rho, vx, vy, vz, P, Gamma_e, Gamma_1, U_aux)."""
        uu = np.zeros(6)
        uu[:len(u)] = u
        w = np.zeros(8)
        c = counts if counts is not None else Counts()
        lib().tref_cons_to_prim(self.h, P(uu), P(w), C.byref(c))
        return w

    def dual_sync(self, U, ids=None, counts=None):
        ids_a = None if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        c = counts if counts is not None else Counts()
        lib().tref_dual_sync(self.h, P(U), 0 if ids_a is None else len(ids_a),
                             None if ids_a is None else IP(ids_a), C.byref(c))
        return c

    def set_phi_sg(self, phi_padded):
        """Self-gravity potential (padded layout, ghosts filled) for the hydro
        sources; None switches it off.  The mesh keeps a reference."""
        self._phi_sg = None if phi_padded is None else np.ascontiguousarray(phi_padded, dtype=np.float64)
        lib().tref_set_phi_sg(self.h, None if self._phi_sg is None else P(self._phi_sg))

    def frame_acceleration(self, U, t, rho_min):
        """(A_fr[3], mass) of Eq. frame-acceleration at time t."""
        A = np.zeros(3)
        mass = np.zeros(1)
        lib().tref_frame_acceleration(self.h, P(U), t, rho_min, P(A), P(mass))
        return A, float(mass[0])

    def boost(self, U, V, rho_min):
        """Galilean boost of Eq. galilean-boost, in place."""
        lib().tref_boost(self.h, P(U), P(np.ascontiguousarray(V, dtype=np.float64)), rho_min)

    def cfl_dt(self, U, cfl, t_b=None):
        dt = np.zeros(self.layout.nb)
        tb = np.zeros(self.layout.nb) if t_b is None else np.ascontiguousarray(t_b, dtype=np.float64)
        lib().tref_cfl_dt(self.h, P(U), cfl, P(tb), P(dt), None)
        return dt

    def step(self, U, dt, t=0.0, scratch=None, counts=None):
        c = counts if counts is not None else Counts()
        S = scratch if scratch is not None else self.new_state()
        lib().tref_step(self.h, P(U), P(S), dt, t, C.byref(c))
        return c

    def lat_factors(self, dt_b, n_lat, merge_frac=0.01):
        f = np.zeros(self.layout.nb, dtype=np.int32)
        dt0 = C.c_double()
        fmax = lib().tref_lat_factors(self.h, P(np.ascontiguousarray(dt_b, dtype=np.float64)), n_lat,
                                      merge_frac, f.ctypes.data_as(i32p), C.byref(dt0))
        return f, dt0.value, fmax

    def lat_window(self, U, f_b, dt0, t=0.0, counts=None):
        c = counts if counts is not None else Counts()
        upd = C.c_int64()
        fb = np.ascontiguousarray(f_b, dtype=np.int32)
        fmax = lib().tref_lat_window(self.h, P(U), fb.ctypes.data_as(i32p), dt0, t, C.byref(c),
                                     C.byref(upd))
        return fmax, upd.value

    def interior(self, U, var=None):
        """Global-grid array [nvar][Nz][Ny][Nx] of the interior cells."""
        return self.layout.to_global(U if var is None else U[var:var + 1])


def riemann(solver, d, dual, wl, wr):
    """a5 on face-state pairs wl, wr [n][8] (rho, vx, vy, vz, P, Gamma_e, Gamma_1,
    U_aux): fluxes [n][6] and face velocities [n]."""
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    n = len(wl)
    F = np.zeros((n, 6))
    vf = np.zeros(n)
    lib().tref_riemann(solver, d, dual, n, P(wl), P(wr), P(F), P(vf))
    return F, vf


def mlp_forward(params, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros_like(x)
    lib().tref_mlp_forward(P(np.ascontiguousarray(params, dtype=np.float64)), len(x), P(x), P(y))
    return y


def mlp_loss_grad(params, x, target):
    x = np.ascontiguousarray(x, dtype=np.float64)
    t = np.ascontiguousarray(target, dtype=np.float64)
    g = np.zeros(MLP_NPARAM)
    loss = lib().tref_mlp_loss_grad(P(np.ascontiguousarray(params, dtype=np.float64)), len(x),
                                    P(x), P(t), P(g))
    return loss, g


def set_num_threads(n):
    lib().tref_set_num_threads(int(n))


def num_threads():
    """Threads the oracle's OpenMP loops use."""
    return int(lib().tref_num_threads())


def mg_solve(src, dx, phi=None, max_cycles=20, tol=0.0, npre=2, npost=2, omega=1.15):
    """Multigrid solve of A_h phi = src on a periodic grid; src [nz][ny][nx].
    Returns (phi, cycles, rms defect)."""
    src = np.ascontiguousarray(src, dtype=np.float64)
    nz, ny, nx = src.shape
    phi = np.zeros_like(src) if phi is None else np.ascontiguousarray(phi, dtype=np.float64).copy()
    d = np.zeros(1)
    dxa = np.ascontiguousarray(dx, dtype=np.float64)
    n = lib().tref_mg_solve(nx, ny, nz, P(dxa), P(src), P(phi), max_cycles, tol, npre, npost, omega, P(d))
    return phi, n, float(d[0])


def mg_solve_bc(src, dx, xmin=(0.0, 0.0, 0.0), isolated=True, lmax=4, centre=None, fmg=True, phi=None,
                max_cycles=20, tol=0.0, npre=2, npost=2, omega=1.15, query=None):
    """Multigrid on a periodic or isolated grid (multipole boundary values), with
    a full-multigrid start.  Returns (phi, cycles, rms defect, rms defect before
    the V-cycles, the expansion at the query points [n][3])."""
    src = np.ascontiguousarray(src, dtype=np.float64)
    nz, ny, nx = src.shape
    phi = np.zeros_like(src) if phi is None else np.ascontiguousarray(phi, dtype=np.float64).copy()
    d, d0 = np.zeros(1), np.zeros(1)
    q = np.zeros((0, 3)) if query is None else np.ascontiguousarray(query, dtype=np.float64).reshape(-1, 3)
    out = np.zeros(len(q))
    c = None if centre is None else np.ascontiguousarray(centre, dtype=np.float64)
    n = lib().tref_mg_solve_bc(nx, ny, nz, P(np.ascontiguousarray(dx, dtype=np.float64)),
                               P(np.ascontiguousarray(xmin, dtype=np.float64)), 1 if isolated else 0, lmax,
                               P(c) if c is not None else None, 1 if fmg else 0, P(src), P(phi), max_cycles, tol,
                               npre, npost, omega, P(d), P(d0), len(q), P(q), P(out))
    return phi, n, float(d[0]), float(d0[0]), out


def mg_prolong(e, nf, isolated=False):
    """The V-cycle's prolongation of a coarse field e [nz][ny][nx] onto a grid of
    nf = (nx, ny, nz) cells (each equal to or twice the coarse count)."""
    e = np.ascontiguousarray(e, dtype=np.float64)
    nc = np.array(e.shape[::-1], dtype=np.int32)
    nfa = np.array(nf, dtype=np.int32)
    out = np.zeros(tuple(nf[::-1]))
    lib().tref_mg_prolong(IP(nfa), IP(nc), 1 if isolated else 0, P(e), P(out))
    return out


def mg_defect(src, phi, dx):
    src = np.ascontiguousarray(src, dtype=np.float64)
    nz, ny, nx = src.shape
    return lib().tref_mg_defect_rms(nx, ny, nz, P(np.ascontiguousarray(dx, dtype=np.float64)), P(src),
                                    P(np.ascontiguousarray(phi, dtype=np.float64)))


def remap(dst, src, Usrc, mode=REMAP_THERMAL, rho_floor=1e-300, u_floor=1e-300):
    """Remap the state Usrc of mesh src onto a new state of mesh dst (Sec. 5.2)."""
    Ud = dst.new_state()
    lib().tref_remap(dst.h, P(Ud), src.h, P(np.ascontiguousarray(Usrc, dtype=np.float64)), mode,
                     rho_floor, u_floor)
    return Ud

