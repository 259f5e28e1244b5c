"""The learned EOS guess on the GPU, through the C ABI: the training kernels'
gradient against the FP64 oracle on the same BF16-rounded weights, the
tensor-core forward pass against the oracle network, training, and the
surrogate inversion against table bisection (identical results by
construction; the acceptance rate is what the network buys)."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = os.path.join(ROOT, "paper_2609_37859_gb300", "data", "eos_saha_hhe_256.npz")
NP = 4482


@pytest.fixture(scope="module")
def tde():
    from paper_2609_37859_gb300 import build, tde as T
    build.build()
    return T


@pytest.fixture(scope="module")
def env(tde, oracle):
    ctx = tde.Context(0)
    eos = tde.EOS.from_file(ctx, TABLE)
    d = np.load(TABLE)
    ot = oracle.EOSTable(int(d["n_rho"]), int(d["n_T"]), tuple(d["lrho"]), tuple(d["lT"]),
                         d["log10_e"], d["log10_P"], d["log10_cs2"])
    return ctx, eos, ot


def bf16_round(w):
    """float32 -> nearest-even BF16, returned as float64."""
    b = np.asarray(w, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def random_weights(seed):
    rng = np.random.default_rng(seed)
    w = np.zeros(NP, dtype=np.float32)
    w[:128] = rng.normal(0, 0.7, 128)
    w[128:192] = rng.normal(0, 0.1, 64)
    w[192:4288] = rng.normal(0, 0.125, 4096)
    w[4288:4352] = rng.normal(0, 0.1, 64)
    w[4352:4480] = rng.normal(0, 0.125, 128)
    w[4480:] = rng.normal(0, 0.1, 2)
    return w


def dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def test_training_gradient_matches_oracle(tde, oracle, env):
    ctx, eos, _ = env
    w = random_weights(1)
    eos.set_weights(w)
    rng = np.random.default_rng(2)
    n = 1000
    x = rng.uniform(-1, 1, (n, 2)).astype(np.float32)
    t = rng.uniform(-1, 1, (n, 2)).astype(np.float32)
    g = torch.zeros(NP, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    eos.grad(dev(x), dev(t), g, loss)
    torch.cuda.synchronize()
    lo, go = oracle.mlp_loss_grad(bf16_round(w), x.astype(np.float64), t.astype(np.float64))
    gg = g.cpu().numpy().astype(np.float64)
    assert float(loss) == pytest.approx(lo, rel=1e-4)
    assert np.linalg.norm(gg - go) <= 1e-3 * np.linalg.norm(go)
    for sl in (slice(0, 128), slice(128, 192), slice(192, 4288), slice(4288, 4352), slice(4352, 4482)):
        assert np.linalg.norm(gg[sl] - go[sl]) <= 2e-3 * np.linalg.norm(go[sl]) + 1e-7


def test_tensor_core_forward_matches_oracle_network(tde, oracle, env):
    ctx, eos, _ = env
    w = random_weights(3)
    eos.set_weights(w)
    rng = np.random.default_rng(4)
    n = 1000   # 8 tiles of 128, ragged tail
    x = rng.uniform(-1, 1, (n, 2)).astype(np.float32)
    y = torch.zeros((n, 2), dtype=torch.float32, device="cuda")
    eos.forward(dev(x), y)
    torch.cuda.synchronize()
    yo = oracle.mlp_forward(bf16_round(w), x.astype(np.float64))
    yg = y.cpu().numpy().astype(np.float64)
    ye, bound = bf16_hidden_emulation(bf16_round(w), x.astype(np.float64))
    # the emulation is the oracle network with the hidden layer rounded to BF16
    assert np.abs(ye - yo).max() < 0.05 * np.abs(yo).max()
    err = np.abs(yg - ye)
    print("tensor-core forward: max |err| %.3e, max err/bound %.3f, mean err/bound %.4f" %
          (err.max(), (err / bound).max(), (err / bound).mean()))
    assert np.all(err <= bound), (err / bound).max()


def bf16_hidden_emulation(w, x):
    """The network as the inference kernel computes it, in FP64: layer 1, SiLU,
    the hidden values rounded to BF16 (the tensor core's operand type), the
    64 x 64 layer, SiLU, layer 3.  Returns the outputs and a per-element
    tolerance of 2^-9 (half a BF16 unit in the last place) of the sum of the
    magnitudes of the output's 65 terms: both sides round the hidden layer to
    BF16; they differ where the SiLU's one-MUFU tanh (relative error about
    2^-11) moves a hidden value across a BF16 rounding midpoint (a change of one
    unit, 2^-7 relative, with random sign, in a few of the 64 terms) and by FP32
    rounding (2^-24 per operation)."""
    H = 64
    W1 = w[:2 * H].reshape(H, 2)
    b1 = w[2 * H:3 * H]
    W2 = w[3 * H:3 * H + H * H].reshape(H, H)
    b2 = w[3 * H + H * H:4 * H + H * H]
    W3 = w[4 * H + H * H:6 * H + H * H].reshape(2, H)
    b3 = w[6 * H + H * H:]
    silu = lambda a: a / (1.0 + np.exp(-a))   # noqa: E731
    h1b = bf16_round(silu(x @ W1.T + b1).astype(np.float32))
    h2 = silu(h1b @ W2.T + b2)
    y = h2 @ W3.T + b3
    return y, 2.0 ** -9 * (np.abs(h2) @ np.abs(W3).T + np.abs(b3))


@pytest.fixture(scope="module")
def trained(tde, env):
    ctx, eos, _ = env
    eos.reset_weights_for_training()
    rep = eos.train(seed=2609, n_samples=1 << 20, epochs=30, batch=4096, lr=3e-3)
    print("training report", rep)
    return rep


def test_training_reduces_loss(trained):
    assert trained["loss_last"] < 0.01 * trained["loss_first"]


def test_surrogate_inversion_equals_bisection(tde, oracle, env, trained):
    ctx, eos, ot = env
    rng = np.random.default_rng(9)
    n = 1 << 16
    lr = rng.uniform(-14, 2, n)
    lT = rng.uniform(2.0, 8.0, n)
    rho = torch.tensor(10 ** lr, dtype=torch.float64, device="cuda")
    T0 = torch.tensor(10 ** lT, dtype=torch.float64, device="cuda")
    e = torch.empty_like(rho)
    eos.eval_rhoT(rho, T0, e=e)
    e[:4] = torch.tensor([-1.0, 1e-40, 1e40, 1e12], dtype=torch.float64)   # clamped inputs
    outs = {}
    for mode in (tde.INVERT_BISECT, tde.INVERT_SURROGATE, tde.INVERT_BISECT_PLAIN):
        T, P, c2 = (torch.empty_like(rho) for _ in range(3))
        before = eos.counts()
        eos.invert(rho, e, T=T, P=P, cs2=c2, mode=mode)
        after = eos.counts()
        outs[mode] = (T.cpu().numpy(), P.cpu().numpy(), c2.cpu().numpy(),
                      after["surrogate_accepted"] - before["surrogate_accepted"])
    for k in range(3):
        assert np.array_equal(outs[tde.INVERT_BISECT][k], outs[tde.INVERT_SURROGATE][k])
        assert np.array_equal(outs[tde.INVERT_BISECT][k], outs[tde.INVERT_BISECT_PLAIN][k])
    acc = outs[tde.INVERT_SURROGATE][3] / n
    print("surrogate acceptance", acc)
    assert acc > 0.5, acc
    # and both equal the oracle's inversion
    idx = rng.integers(0, n, 300)
    ec = e.cpu().numpy()
    rc = rho.cpu().numpy()
    for q in idx:
        want = ot.invert(rc[q], ec[q])
        assert outs[tde.INVERT_SURROGATE][0][q] == pytest.approx(want[0], rel=1e-12)
        assert outs[tde.INVERT_SURROGATE][1][q] == pytest.approx(want[1], rel=1e-12)


def test_what_training_buys(tde, oracle, env, trained):
    """The gain of the trained network over the method without it: on the same
    inputs (the EOS-inversion workload's recombination band), the share of cells
    whose Newton step from the guess lands in the bracketing temperature cell
    (they skip the table search) with the trained weights and with two sets of
    untrained (random) weights; the results equal bisection in every case (the
    acceptance is what the network buys, never the answer)."""
    ctx, eos, _ = env
    w_trained = eos.get_weights()
    from paper_2609_37859_gb300 import workloads as wl
    n = 1 << 18
    g = torch.Generator(device="cuda")
    g.manual_seed(12)
    rho, T0 = wl.c3_inputs(n, g, "cuda")
    e = torch.empty_like(rho)
    eos.eval_rhoT(rho, T0, e=e)
    Tb, Pb = torch.empty_like(rho), torch.empty_like(rho)
    eos.invert(rho, e, T=Tb, P=Pb, mode=tde.INVERT_BISECT)

    def acceptance():
        T, P = torch.empty_like(rho), torch.empty_like(rho)
        before = eos.counts()["surrogate_accepted"]
        eos.invert(rho, e, T=T, P=P, mode=tde.INVERT_SURROGATE)
        torch.cuda.synchronize()
        assert torch.equal(T, Tb) and torch.equal(P, Pb)
        return (eos.counts()["surrogate_accepted"] - before) / n

    try:
        acc_trained = acceptance()
        eos.set_weights(random_weights(5))
        acc_random = acceptance()
        eos.set_weights(random_weights(6))
        acc_random2 = acceptance()
    finally:
        eos.set_weights(w_trained)
    print("acceptance trained %.3f, untrained %.3f / %.3f" % (acc_trained, acc_random, acc_random2))
    # measured on GB300 after 30 epochs: 0.67 trained, 0.34 / 0.29 untrained (the
    # landing cell of one Newton step is often right even from a poor guess where
    # the column is nearly linear; the recombination band is where training pays)
    assert acc_trained > 0.6
    assert acc_trained > max(acc_random, acc_random2) + 0.25
    assert acceptance() == acc_trained   # the trained weights are back


def test_expired_wait_is_reported_and_results_stand(tde, oracle, env, trained):
    """Failure detection without a fault: the test hook makes the inference issue
    no tensor-core work, so its bounded wait for the results expires; the kernel
    sets the status word and returns, tde_eos_check reports TDE_ETIMEOUT once, the
    cells take the bisection fallback (results identical to bisection) and the
    context stays usable."""
    ctx, eos, _ = env
    rng = np.random.default_rng(77)
    n = 4096
    rho = torch.tensor(10 ** rng.uniform(-14, 2, n), dtype=torch.float64, device="cuda")
    T0 = torch.tensor(10 ** rng.uniform(3.4, 5.4, n), dtype=torch.float64, device="cuda")
    e = torch.empty_like(rho)
    eos.eval_rhoT(rho, T0, e=e)
    Tb, Pb = torch.empty_like(rho), torch.empty_like(rho)
    eos.invert(rho, e, T=Tb, P=Pb, mode=tde.INVERT_BISECT)
    eos.check()   # nothing pending
    T, P = torch.empty_like(rho), torch.empty_like(rho)
    eos.inject_wait_expiry(True)
    try:
        eos.invert(rho, e, T=T, P=P, mode=tde.INVERT_SURROGATE)
        with pytest.raises(tde.TDEError) as ei:
            eos.check()
        assert ei.value.code == tde.TDE_ETIMEOUT
    finally:
        eos.inject_wait_expiry(False)
    assert torch.equal(T, Tb) and torch.equal(P, Pb)
    eos.check()   # the flag was cleared by the report
    before = eos.counts()["surrogate_accepted"]
    eos.invert(rho, e, T=T, P=P, mode=tde.INVERT_SURROGATE)
    eos.check()
    assert torch.equal(T, Tb) and torch.equal(P, Pb)
    assert eos.counts()["surrogate_accepted"] - before > n // 2
