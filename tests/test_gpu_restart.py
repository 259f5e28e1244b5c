"""Checkpoint and resume: the state is the caller's device array, so a restart is
that array written to a raw .npy file with the mesh time (and, for the learned
closure, the network's weights), then loaded into a new context, EOS and mesh.
The restarted run reproduces the continued run bit for bit: synchronised steps
with the moving point mass and excision, then a LAT window under the learned-guess
closure."""
import numpy as np
import pytest

from paper_2609_37859_gb300 import workloads as wl
from test_gpu_hydro import Pair, SCHEME_KEYS, TABLE_FILE  # noqa: F401

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_hydro import tde, ctx, tables  # noqa: E402,F401


def test_restart_reproduces_the_continued_run_bitwise(oracle, tde, ctx, tables, tmp_path):
    ot, eos = tables
    eos.reset_weights_for_training()
    eos.train(seed=7, n_samples=1 << 16, epochs=4, batch=4096, lr=3e-3)
    rho0, v0 = 0.7382, 1.0948e8
    lay = wl.mixed_layout((16, 16, 8), 8, {(0, 0, 0)}, ((-2.0, 2.0), (-2.0, 2.0), (-1.0, 1.0)), (0, 0, 0), 3)
    x, y, z = lay.cell_centres()
    r = np.sqrt(x ** 2 + y ** 2 + z ** 2)
    rho = 1e-6 + 1e-3 * np.exp(-((r - 1.0) / 0.3) ** 2)
    Pc = rho * rho0 * 1.380649e-16 * 1e4 / (0.6 * 1.6605e-24) / (rho0 * v0 * v0)
    W = wl.prim_state(lay, rho, -y * 0.3, x * 0.3, 0 * rho, Pc)
    bh = dict(on=1, excise=1, GM=1000 / (4 * np.pi), r_soft=0.005, r_exc=0.35, x0=(0.05, -0.02, 0.0),
              v0=(0.1, 0.0, 0.0))
    scheme = dict(eos=1, recon=1, dual=1, eta1=1e-3, eta2=1e-4, rho_floor=1e-10, p_floor=1e-16,
                  u_floor=1.5e-16, unit_rho=rho0, unit_e=v0 * v0)
    A = Pair(oracle, tde, ctx, lay, W, tables, bh=bh, **scheme)
    params = tde.make_params(eos_mode=tde.INVERT_SURROGATE, **{k: v for k, v in scheme.items() if k in SCHEME_KEYS})
    A.gm.set_params(params)
    A.gm.set_time(0.0)
    for _ in range(3):
        A.gm.step(cfl=0.3, bh=A.bh)
    # checkpoint: the state, the time, the network
    np.save(tmp_path / "U.npy", A.gpu("U"))
    np.save(tmp_path / "w.npy", eos.get_weights())
    t_ck = A.gm.get_time()

    def advance(mesh, bhs):
        for _ in range(2):
            mesh.step(cfl=0.3, bh=bhs)
        f, dt0, fmax = mesh.lat_assign(3, 0.3, merge_frac=0.0, bh=bhs)
        mesh.lat_window(bh=bhs, use_graph=True)
        torch.cuda.synchronize()
        return mesh.U.cpu().numpy(), mesh.get_time(), f

    A.gm.counts(reset=True)
    UA, tA, fA = advance(A.gm, A.bh)
    cA = A.gm.counts()
    # resume in a new context, EOS and mesh
    ctx2 = tde.Context(0)
    eos2 = tde.EOS.from_file(ctx2, TABLE_FILE)
    eos2.set_weights(np.load(tmp_path / "w.npy"))
    m2 = tde.Mesh(ctx2, lay, params, eos2)
    m2.U.copy_(torch.from_numpy(np.load(tmp_path / "U.npy")))
    m2.set_time(t_ck)
    UB, tB, fB = advance(m2, A.bh)
    cB = m2.counts()
    assert np.array_equal(fA, fB) and len(np.unique(fA)) > 1
    assert tA == tB
    assert np.array_equal(UA, UB)
    # the same decisions, and the restored network accepts the same cells
    assert cA == cB and cA["surrogate_accepted"] > 0 and cA["excised"] > 0
