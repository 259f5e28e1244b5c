"""Seeded synthetic workloads: MeshBlock layouts and primitive initial fields.

This module holds geometry, random numbers and closed-form primitive profiles
only -- none of the hydro method's arithmetic.  The conversion of primitives to
conserved variables (which needs the equation of state) is done separately by
the CUDA library (``tde_prim_to_cons``) and by the CPU oracle, each with its own
code.  Thermodynamic constants a profile needs (a pressure level, a sound speed)
are passed in by the caller.

State layout shared by every consumer: a state is ``[nvar][ntot]`` float64 with
MeshBlock ``b`` occupying padded cells ``off[b] .. off[b+1]``, padded index
``(k * Py + j) * Px + i`` (x fastest), interior cells starting at ``ng`` in
every active direction (a direction with one global cell is inactive and has no
ghost cells).
"""
from dataclasses import dataclass, field

import numpy as np

OUTFLOW, PERIODIC = 0, 1


@dataclass
class MeshLayout:
    blocks: np.ndarray          # [nb, 6] int32: i0, j0, k0, nx, ny, nz
    N: tuple                    # global cells per direction
    xmin: tuple
    dx: tuple
    bc: tuple                   # OUTFLOW / PERIODIC per direction
    ng: int
    levels: np.ndarray = None   # [nb] refinement level per block (None: all 0)
    off: np.ndarray = field(init=False)
    pd: np.ndarray = field(init=False)

    def __post_init__(self):
        self.blocks = np.ascontiguousarray(self.blocks, dtype=np.int32).reshape(-1, 6)
        if self.levels is not None:
            self.levels = np.ascontiguousarray(self.levels, dtype=np.int32).reshape(-1)
            if not self.levels.any():
                self.levels = None
        act = np.array([n > 1 for n in self.N])
        self.active = act
        self.pd = self.blocks[:, 3:6] + 2 * self.ng * act[None, :]
        sizes = self.pd.prod(axis=1).astype(np.int64)
        self.off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)

    @property
    def nb(self):
        return len(self.blocks)

    @property
    def ntot(self):
        return int(self.off[-1])

    @property
    def ncells(self):
        return int(np.prod(self.N))

    def gofs(self, a):
        return self.ng if self.active[a] else 0

    def interior_index(self, b):
        """(flat padded indices into the state, global (gk, gj, gi)) of block b's interior."""
        i0, j0, k0, nx, ny, nz = self.blocks[b]
        px, py, _ = self.pd[b]
        gx, gy, gz = self.gofs(0), self.gofs(1), self.gofs(2)
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        flat = self.off[b] + ((k + gz) * py + (j + gy)) * px + (i + gx)
        return flat, (k + k0, j + j0, i + i0)

    def to_global(self, U):
        """[nvar, ntot] state -> [nvar, Nz, Ny, Nx] interior grid."""
        U = np.asarray(U)
        out = np.zeros((U.shape[0], self.N[2], self.N[1], self.N[0]), dtype=U.dtype)
        for b in range(self.nb):
            flat, (gk, gj, gi) = self.interior_index(b)
            out[:, gk, gj, gi] = U[:, flat]
        return out

    def from_global(self, G):
        """[nvar, Nz, Ny, Nx] -> [nvar, ntot] state (ghost cells zero)."""
        G = np.asarray(G)
        U = np.zeros((G.shape[0], self.ntot), dtype=G.dtype)
        for b in range(self.nb):
            flat, (gk, gj, gi) = self.interior_index(b)
            U[:, flat] = G[:, gk, gj, gi]
        return U

    def level(self, b):
        return 0 if self.levels is None else int(self.levels[b])

    def block_dx(self, b):
        L = self.level(b)
        return tuple(self.dx[a] / (1 << L) if self.active[a] else self.dx[a] for a in range(3))

    def interior_flat(self):
        """Flat padded indices of every interior cell, block by block."""
        return np.concatenate([self.interior_index(b)[0].ravel() for b in range(self.nb)])

    def interior_centres(self):
        """x, y, z and cell volume of every interior cell, in interior_flat() order."""
        xs, ys, zs, vs = [], [], [], []
        for b in range(self.nb):
            _, (gk, gj, gi) = self.interior_index(b)
            d = self.block_dx(b)
            xs.append((self.xmin[0] + (gi.ravel() + 0.5) * d[0]))
            ys.append((self.xmin[1] + (gj.ravel() + 0.5) * d[1]))
            zs.append((self.xmin[2] + (gk.ravel() + 0.5) * d[2]))
            vs.append(np.full(gi.size, d[0] * d[1] * d[2]))
        return np.concatenate(xs), np.concatenate(ys), np.concatenate(zs), np.concatenate(vs)

    def state_from_cells(self, F):
        """[nvar, n_interior] values in interior_flat() order -> [nvar, ntot] state."""
        F = np.asarray(F)
        U = np.zeros((F.shape[0], self.ntot), dtype=F.dtype)
        U[:, self.interior_flat()] = F
        return U

    def cell_centres(self):
        """x, y, z of the global interior grid, each [Nz, Ny, Nx]."""
        ax = [self.xmin[a] + (np.arange(self.N[a]) + 0.5) * self.dx[a] for a in range(3)]
        z, y, x = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return x, y, z


def uniform_layout(N, block, domain=((0.0, 1.0),) * 3, bc=(OUTFLOW,) * 3, ng=2):
    """Uniform grid of N[a] cells per direction split into blocks of block[a] cells
    (the last block of a direction takes the remainder: ragged tails allowed)."""
    starts = []
    for a in range(3):
        s = list(range(0, N[a], block[a]))
        starts.append([(x, min(block[a], N[a] - x)) for x in s])
    blocks = []
    for k0, nz in starts[2]:
        for j0, ny in starts[1]:
            for i0, nx in starts[0]:
                blocks.append((i0, j0, k0, nx, ny, nz))
    dx = tuple((domain[a][1] - domain[a][0]) / N[a] for a in range(3))
    return MeshLayout(np.array(blocks), tuple(N), tuple(d[0] for d in domain), dx, tuple(bc), ng)


def mixed_layout(root_N, root_block, split, domain, bc, ng):
    """Uniform-cell grid of root blocks; the root blocks whose index is in `split`
    are replaced by eight half-size blocks (same cell size, no refinement)."""
    nbx = [root_N[a] // root_block for a in range(3)]
    blocks = []
    h = root_block // 2
    for bk in range(nbx[2]):
        for bj in range(nbx[1]):
            for bi in range(nbx[0]):
                i0, j0, k0 = bi * root_block, bj * root_block, bk * root_block
                if (bi, bj, bk) in split:
                    for dk in (0, h):
                        for dj in (0, h):
                            for di in (0, h):
                                blocks.append((i0 + di, j0 + dj, k0 + dk, h, h, h))
                else:
                    blocks.append((i0, j0, k0, root_block, root_block, root_block))
    dx = tuple((domain[a][1] - domain[a][0]) / root_N[a] for a in range(3))
    return MeshLayout(np.array(blocks), tuple(root_N), tuple(d[0] for d in domain), dx, tuple(bc), ng)


def smr_layout(root_N, block, domain, bc, ng, refine, max_level):
    """Statically refined mesh: root blocks of `block` cells (a multiple of 4 per
    active direction) on the level-0 grid of root_N cells; a block of level L < max_level
    whose region meets refine(lo, hi, L) (lo, hi: its corners) is split into 2^d
    children of the same cell count on level L + 1; then blocks are split until the
    mesh is 2:1 balanced across faces, edges and corners (periodic images included)."""
    act = [n > 1 for n in root_N]
    dx0 = tuple((domain[a][1] - domain[a][0]) / root_N[a] for a in range(3))
    bs = [block[a] if act[a] else 1 for a in range(3)]
    blocks = []
    for k0 in range(0, root_N[2], bs[2]):
        for j0 in range(0, root_N[1], bs[1]):
            for i0 in range(0, root_N[0], bs[0]):
                blocks.append((0, i0, j0, k0))

    def corners(blk):
        L, i0, j0, k0 = blk
        lo, hi = [], []
        for a, o in enumerate((i0, j0, k0)):
            d = dx0[a] / (1 << L) if act[a] else dx0[a]
            lo.append(domain[a][0] + o * d)
            hi.append(domain[a][0] + (o + bs[a]) * d)
        return lo, hi

    def children(blk):
        L, i0, j0, k0 = blk
        out = []
        for dk in (range(2) if act[2] else (0,)):
            for dj in (range(2) if act[1] else (0,)):
                for di in (range(2) if act[0] else (0,)):
                    o = [2 * i0 + di * bs[0], 2 * j0 + dj * bs[1], 2 * k0 + dk * bs[2]]
                    out.append((L + 1, *[o[a] if act[a] else 0 for a in range(3)]))
        return out

    for L in range(max_level):
        nxt = []
        for blk in blocks:
            if blk[0] == L and refine(*corners(blk), L):
                nxt.extend(children(blk))
            else:
                nxt.append(blk)
        blocks = nxt
    # 2:1 balance on the finest lattice
    while True:
        lmax = max(b[0] for b in blocks)
        NF = [root_N[a] << lmax if act[a] else 1 for a in range(3)]
        own = np.full(NF[::-1], -1, dtype=np.int64)
        for q, (L, i0, j0, k0) in enumerate(blocks):
            s = lmax - L
            sl = []
            for a, o in zip((2, 1, 0), (k0, j0, i0)):
                if act[a]:
                    sl.append(slice(o << s, (o + bs[a]) << s))
                else:
                    sl.append(slice(0, 1))
            own[tuple(sl)] = q
        lev = np.array([b[0] for b in blocks])
        split = set()
        for q, (L, i0, j0, k0) in enumerate(blocks):
            s = lmax - L
            idx = []
            for a, o in zip((2, 1, 0), (k0, j0, i0)):
                if not act[a]:
                    idx.append(np.array([0]))
                    continue
                r = np.arange((o - 1) << s, (o + bs[a] + 1) << s)
                if bc[a] == PERIODIC:
                    r = r % NF[a]
                else:
                    r = np.clip(r, 0, NF[a] - 1)
                idx.append(r)
            nb_lev = lev[own[np.ix_(*idx)]]
            if nb_lev.max() > L + 1:
                split.add(q)
        if not split:
            break
        nxt = []
        for q, blk in enumerate(blocks):
            nxt.extend(children(blk) if q in split else [blk])
        blocks = nxt
    arr = np.array([(i0, j0, k0, bs[0], bs[1], bs[2]) for (L, i0, j0, k0) in blocks], dtype=np.int32)
    lev = np.array([b[0] for b in blocks], dtype=np.int32)
    return MeshLayout(arr, tuple(root_N), tuple(d[0] for d in domain), dx0, tuple(bc), ng, lev)


def prim_cells(layout, rho, vx, vy, vz, P):
    """Pack per-cell primitive values (interior_flat() order) into the padded layout."""
    F = np.stack([np.broadcast_to(np.asarray(f, dtype=np.float64), (layout.interior_flat().size,))
                  for f in (rho, vx, vy, vz, P)])
    return layout.state_from_cells(F)


def prim_state(layout, rho, vx, vy, vz, P):
    """Pack global [Nz, Ny, Nx] primitive fields into the padded layout, 5 fields."""
    G = np.stack([np.broadcast_to(np.asarray(f, dtype=np.float64), (layout.N[2], layout.N[1], layout.N[0]))
                  for f in (rho, vx, vy, vz, P)])
    return layout.from_global(G)


# --------------------------------------------------------------------- profiles

def sod(layout, axis=0, rho=(1.0, 0.125), P=(1.0, 0.1), x0=0.5):
    """Sod shock tube along `axis` (rho 1/0.125, P 1/0.1, at rest)."""
    c = layout.cell_centres()[axis]
    left = c < x0
    r = np.where(left, rho[0], rho[1])
    p = np.where(left, P[0], P[1])
    z = np.zeros_like(r)
    return prim_state(layout, r, z, z, z, p)


def sound_wave(layout, amp=1e-6, rho0=1.0, P0=None, gamma=5.0 / 3.0, axis=0, wavelength=1.0):
    """Linear right-moving sound wave; rho0, P0 background, c_s = sqrt(gamma P0 / rho0)."""
    P0 = 1.0 / gamma if P0 is None else P0
    cs = np.sqrt(gamma * P0 / rho0)
    x = layout.cell_centres()[axis]
    s = np.sin(2 * np.pi * (x - layout.xmin[axis]) / wavelength)
    r = rho0 * (1 + amp * s)
    v = cs * amp * s
    p = P0 * (1 + gamma * amp * s)
    z = np.zeros_like(r)
    vel = [z, z, z]
    vel[axis] = v
    return prim_state(layout, r, *vel, p)


def entropy_wave(layout, rho0, P0, v_adv, amp=1e-3, seed=0, axis=0, wavelength=1.0):
    """Entropy wave rho = rho0 (1 + amp sin(2 pi x / wavelength + phi)), uniform P and v
    along `axis`; phi drawn from the seed."""
    phi = np.random.default_rng(seed).uniform(0.0, 2 * np.pi)
    x = layout.cell_centres()[axis]
    r = rho0 * (1 + amp * np.sin(2 * np.pi * (x - layout.xmin[axis]) / wavelength + phi))
    z = np.zeros_like(r)
    vel = [z, z, z]
    vel[axis] = np.full_like(r, v_adv)
    return prim_state(layout, r, *vel, np.full_like(r, P0)), phi


def random_smooth(layout, seed=0, rho0=1.0, P0=1.0, drho=0.2, dv=0.3, dP=0.2, modes=3):
    """Seeded smooth periodic fields (sums of low Fourier modes)."""
    rng = np.random.default_rng(seed)
    x, y, z = layout.cell_centres()
    L = [layout.dx[a] * layout.N[a] for a in range(3)]

    def field_(amp):
        f = np.zeros_like(x)
        for _ in range(modes):
            k = rng.integers(0, 3, size=3)
            ph = rng.uniform(0, 2 * np.pi)
            f += np.sin(2 * np.pi * (k[0] * x / L[0] + k[1] * y / L[1] + k[2] * z / L[2]) + ph)
        return amp * f / modes

    r = rho0 * (1 + field_(drho))
    return prim_state(layout, r, field_(dv), field_(dv), field_(dv), P0 * (1 + field_(dP)))


# ------------------------------------------------------------ stream (C4) ---

# code units of Table 1: M0 = 1 Msun, L0 = 2 Rsun, t0 = 1270.9 s, G = 1 / (4 pi)
RHO0_CGS, V0_CGS = 0.7382, 1.0948e8
G_CODE = 1.0 / (4.0 * np.pi)
RSUN_CODE = 0.5


def stream_c4(split_nearest=16, n_root=(10, 10, 4), block=32, ng=3, rp_rsun=10.0, ra_rsun=28.0,
              sigma_rsun=1.0, rho_peri=1e-2, rho_apo=1e-10, rho_amb=1e-14, mach_max=1e3,
              m_bh=1000.0, mu=1.3, gamma=5.0 / 3.0):
    """Cold thin stream on an ellipse around a point mass (the LAT workload).

    Domain x, y in [-32, 32] Rsun, z in [-12.8, 12.8] Rsun (code units of
    Table 1), cells of 0.2 Rsun; root blocks of `block`^3, the `split_nearest`
    root blocks closest to pericentre split into eight half-size blocks.  A
    Gaussian tube (sigma) follows the ellipse with the BH at its focus
    (pericentre rp, apocentre ra); its centre density falls log-linearly in the
    orbital phase from rho_peri to rho_apo (g/cm^3); the gas moves on the
    Keplerian ellipse; one temperature makes the fastest cell Mach mach_max for
    an ideal-gas sound speed with mean molecular weight mu (the caller turns
    (rho, T) into pressure with its EOS).  Returns (layout, fields) with fields a
    dict of global arrays rho (code units), vx, vy, vz (code units), T (K), and
    the BH parameters."""
    N = (n_root[0] * block, n_root[1] * block, n_root[2] * block)
    half = (32.0 * RSUN_CODE, 32.0 * RSUN_CODE, 12.8 * RSUN_CODE)
    domain = tuple((-h, h) for h in half)
    rp, ra = rp_rsun * RSUN_CODE, ra_rsun * RSUN_CODE
    a_orb = 0.5 * (rp + ra)
    ecc = (ra - rp) / (ra + rp)
    # root blocks nearest to pericentre (at +x)
    centres = []
    dx = tuple((domain[a][1] - domain[a][0]) / N[a] for a in range(3))
    for bk in range(n_root[2]):
        for bj in range(n_root[1]):
            for bi in range(n_root[0]):
                c = [domain[0][0] + (bi + 0.5) * block * dx[0], domain[1][0] + (bj + 0.5) * block * dx[1],
                     domain[2][0] + (bk + 0.5) * block * dx[2]]
                centres.append(((c[0] - rp) ** 2 + c[1] ** 2 + c[2] ** 2, (bi, bj, bk)))
    centres.sort()
    split = {c[1] for c in centres[:split_nearest]}
    lay = mixed_layout(N, block, split, domain, (0, 0, 0), ng)
    x, y, z = lay.cell_centres()
    # distance to the ellipse r(phi) = a (1 - e^2) / (1 + e cos phi), sampled
    # densely, on the (x, y) plane (it does not depend on z)
    phi = np.linspace(-np.pi, np.pi, 4097)
    rr = a_orb * (1 - ecc ** 2) / (1 + ecc * np.cos(phi))
    pts = np.stack([rr * np.cos(phi), rr * np.sin(phi)], axis=1)
    flat = np.stack([x[0].ravel(), y[0].ravel()], axis=1)
    best_d2 = np.full(flat.shape[0], np.inf)
    best_k = np.zeros(flat.shape[0], dtype=np.int64)
    for k0 in range(0, len(pts), 32):
        chunk = pts[k0:k0 + 32]
        d2 = ((flat[:, None, :] - chunk[None, :, :]) ** 2).sum(axis=2)
        kk = np.argmin(d2, axis=1)
        dd = d2[np.arange(len(kk)), kk]
        upd = dd < best_d2
        best_d2[upd] = dd[upd]
        best_k[upd] = kk[upd] + k0
    best_d2 = np.broadcast_to(best_d2.reshape(x.shape[1:]), x.shape)
    best_k = np.broadcast_to(best_k.reshape(x.shape[1:]), x.shape)
    best_d2 = best_d2 + z ** 2
    ph = phi[best_k]
    frac = np.abs(ph) / np.pi                      # 0 at pericentre, 1 at apocentre
    lrho_c = np.log10(rho_peri) + frac * (np.log10(rho_apo) - np.log10(rho_peri))
    sig = sigma_rsun * RSUN_CODE
    tube = np.exp(-0.5 * best_d2 / sig ** 2)
    rho_cgs = rho_amb + (10.0 ** lrho_c) * tube
    # Keplerian speed on the ellipse, direction tangent (counter-clockwise)
    GM = G_CODE * m_bh
    rloc = a_orb * (1 - ecc ** 2) / (1 + ecc * np.cos(ph))
    vmag = np.sqrt(GM * (2.0 / rloc - 1.0 / a_orb))
    # tangent of the ellipse at phi: d/dphi (r cos phi, r sin phi)
    drdphi = a_orb * (1 - ecc ** 2) * ecc * np.sin(ph) / (1 + ecc * np.cos(ph)) ** 2
    tx = drdphi * np.cos(ph) - rloc * np.sin(ph)
    ty = drdphi * np.sin(ph) + rloc * np.cos(ph)
    tn = np.sqrt(tx ** 2 + ty ** 2)
    w = np.clip(tube * 4.0, 0.0, 1.0)               # gas in the tube moves, ambient at rest
    vx, vy = w * vmag * tx / tn, w * vmag * ty / tn
    vmax = float(np.max(np.sqrt(vx ** 2 + vy ** 2)))
    cs = vmax * V0_CGS / mach_max
    kB, mu_m = 1.380649e-16, mu * 1.66053906660e-24
    T = np.full(x.shape, cs * cs * mu_m / (gamma * kB))
    fields = {"rho": rho_cgs / RHO0_CGS, "vx": vx, "vy": vy, "vz": np.zeros_like(vx), "T": T}
    bh = {"GM": GM, "r_soft": 0.01 * RSUN_CODE, "r_exc": 0.4 * RSUN_CODE, "x0": (0.0, 0.0, 0.0)}
    return lay, fields, bh


def lane_emden(n=1.5, h=1e-3):
    """Lane-Emden function theta(xi) of index n by fourth-order Runge-Kutta from
    the series start at small xi; returns (xi, theta, xi_1, -xi_1^2 theta'(xi_1))."""
    xi0 = 1e-4
    y = np.array([1.0 - xi0 ** 2 / 6.0, -xi0 / 3.0])

    def f(x, v):
        th = max(v[0], 0.0)
        return np.array([v[1], -th ** n - 2.0 * v[1] / x])
    xs, ths = [xi0], [y[0]]
    x = xi0
    while y[0] > 0.0:
        k1 = f(x, y)
        k2 = f(x + h / 2, y + h / 2 * k1)
        k3 = f(x + h / 2, y + h / 2 * k2)
        k4 = f(x + h, y + h * k3)
        y_new = y + h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
        if y_new[0] <= 0.0:   # linear interpolation to the surface
            t = y[0] / (y[0] - y_new[0])
            x1 = x + t * h
            dth = y[1] + t * (y_new[1] - y[1])
            xs.append(x1)
            ths.append(0.0)
            return np.array(xs), np.array(ths), x1, -x1 * x1 * dth
        x += h
        y = y_new
        xs.append(x)
        ths.append(y[0])
    raise RuntimeError("Lane-Emden integration did not reach the surface")


def star_c5(n_blocks=(16, 16, 8), block=32, ng=3, half_rsun=(16.0, 16.0, 8.0), stretch=4.0,
            star_at_rsun=(0.0, 0.0), m_star=1.0, r_star_rsun=1.0, m_bh=1000.0,
            bh_at_rsun=(12.0, 10.0, 0.0), shear=0.1, rho_floor=1e-10, p_floor=1e-12,
            inflow_rsun=4.0, seed=0):
    """Production-shaped workload: an n = 1.5 polytrope (m_star, r_star) stretched
    along x into an ellipsoid (long semi-axis stretch * R, the other two
    R / sqrt(stretch): volume and mass kept), in the frame that moves with the
    star (the paper's runs start in such a translating frame): the gas carries
    only a seeded linear velocity gradient along the long axis, and the point
    mass m_bh passes at the parabolic speed for its initial distance, moving
    along -x.  The ambient is the floor state of Table 1 (rho_floor, p_floor in
    code units); within inflow_rsun of the point mass it moves with it and falls
    in at the free-fall speed.  Code units of Table 1 (length 2 Rsun, mass 1 Msun,
    G = 1/(4 pi)).  Uniform grid of n_blocks blocks of `block`^3 cells on x, y in
    [-half, half] and z in [-half_z, half_z] Rsun.  Returns (layout, fields, bh)
    with fields the global arrays rho, vx, vy, vz, P (code units) and bh the point
    mass (position, velocity, softening, excision radius)."""
    rng = np.random.default_rng(seed)
    N = tuple(n_blocks[a] * block for a in range(3))
    domain = tuple((-h * RSUN_CODE, h * RSUN_CODE) for h in half_rsun)
    lay = uniform_layout(N, (block, block, block), domain, (0, 0, 0), ng)
    x, y, z = lay.cell_centres()
    xi, th, xi1, mass_c = lane_emden(1.5)
    R = r_star_rsun * RSUN_CODE
    alpha = R / xi1
    rho_c = m_star / (4.0 * np.pi * alpha ** 3 * mass_c)          # code units
    P_c = 4.0 * np.pi * G_CODE * alpha ** 2 * rho_c ** 2 / 2.5     # (n + 1) = 2.5
    a_l, a_t = stretch * R, R / np.sqrt(stretch)
    xs, ys = (c * RSUN_CODE for c in star_at_rsun)
    xp, yp = x - xs, y - ys
    re = np.sqrt((xp / a_l) ** 2 + (yp / a_t) ** 2 + (z / a_t) ** 2)   # 1 at the surface
    inside = re < 1.0
    thv = np.where(inside, np.interp(np.minimum(re, 1.0) * xi1, xi, th), 0.0)
    rho = rho_floor + rho_c * thv ** 1.5
    P = p_floor + P_c * thv ** 2.5
    GM = G_CODE * m_bh
    bx = tuple(c * RSUN_CODE for c in bh_at_rsun)
    r0 = np.hypot(xs - bx[0], ys - bx[1])
    v_c = np.sqrt(2.0 * GM / r0)                                   # parabolic speed
    kappa = rng.uniform(0.5, 1.0) * shear * v_c / a_l              # seeded shear rate
    w = np.clip(thv * 20.0, 0.0, 1.0)                              # the star's gas only
    vx = w * kappa * xp
    vy = np.zeros_like(vx)
    vz = np.zeros_like(vx)
    # floor gas near the point mass already falls in (radially in its frame,
    # free-fall speed of the softened potential, blended to rest at r_in), so the
    # run starts from the quasi-steady inflow instead of its transient
    rx, ry, rz = x - bx[0], y - bx[1], z - bx[2]
    r = np.sqrt(rx ** 2 + ry ** 2 + rz ** 2)
    r_in = inflow_rsun * RSUN_CODE
    r_s = 0.01 * RSUN_CODE
    u_ff = np.sqrt(2.0 * GM * np.maximum(1.0 / np.sqrt(r ** 2 + r_s ** 2) - 1.0 / np.sqrt(r_in ** 2 + r_s ** 2), 0.0))
    blend = np.where(r < r_in, 1.0 - w, 0.0)
    u = np.where(r < r_in, u_ff, 0.0) * blend
    rr = np.maximum(r, 1e-30)
    vx += blend * (-v_c) - u * rx / rr
    vy += -u * ry / rr
    vz += -u * rz / rr
    fields = {"rho": rho, "vx": vx, "vy": vy, "vz": vz, "P": P}
    bh = {"GM": GM, "r_soft": 0.01 * RSUN_CODE, "r_exc": 0.4 * RSUN_CODE, "x0": bx,
          "v0": (-v_c, 0.0, 0.0), "v_star": v_c, "rho_c": rho_c, "P_c": P_c}
    return lay, fields, bh


# ------------------------------------------------ EOS-inversion inputs (C3) ---

C3_BAND_FILE = __import__("os").path.join(__import__("os").path.dirname(__import__("os").path.abspath(__file__)),
                                          "data", "c3_recombination_band.npz")


def c3_inputs(n, generator, device):
    """Inputs of the EOS-inversion workload, on the device: log10 rho ~ U[-14, 2]
    g/cm^3 and log10 T ~ U[T_lo(rho), T_hi(rho)], the band from 1 % ionised
    hydrogen to 99 % He2+ (a data file written from the oracle's Saha solver at 257
    densities; linear in log10 rho in between).  Returns (rho, T) in cgs, float64
    torch tensors drawn from `generator`."""
    import torch
    d = np.load(C3_BAND_FILE)
    lrho = d["lrho"]
    lo_t = torch.tensor(d["lT_lo"], dtype=torch.float64, device=device)
    hi_t = torch.tensor(d["lT_hi"], dtype=torch.float64, device=device)
    lr = torch.rand(n, generator=generator, device=device, dtype=torch.float64) * 16.0 - 14.0
    x = (lr - lrho[0]) / (lrho[-1] - lrho[0]) * (len(lrho) - 1)
    i = x.floor().clamp(0, len(lrho) - 2).long()
    w = x - i
    lo = lo_t[i] * (1 - w) + lo_t[i + 1] * w
    hi = hi_t[i] * (1 - w) + hi_t[i + 1] * w
    u = torch.rand(n, generator=generator, device=device, dtype=torch.float64)
    lT = lo + u * (hi - lo)
    return torch.pow(10.0, lr), torch.pow(10.0, lT)
