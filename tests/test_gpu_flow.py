"""GPU learned importance sampler (BF16 tensor-core coupling flow) against the
FP64 reference of oracle/flow_ref.py, through the C ABI.

* The identity initialisation maps u to itself with log-Jacobian 0.
* A random flow agrees with the reference evaluated with the same (BF16-rounded)
  hidden weights; the residual is the BF16 rounding of the hidden activations.
* Whatever the rounding inside the MLPs, the map's log-Jacobian is exact, so
  E_u |dy/du| = 1 (the sampling density integrates to one).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
D, C, H, K = 7, 16, 128, 6


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from oracle import flow_ref as F
    from paper_1407_7595_gb300 import abi
    abi.lib()
    return torch, abi, F


def bf16(torch, a):
    return torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()


def test_param_layout(env):
    torch, abi, F = env
    layers = F.init_params(D, K, H, C, seed=1, zero_last=False)
    flat = F.to_flat(layers)
    assert flat.size == abi.mem_flow_param_count()
    f = abi.mem_flow_create(7)
    abi.mem_flow_set_params(f, flat)
    back = abi.mem_flow_get_params(f)
    assert np.array_equal(back, flat.astype(np.float32))
    abi.mem_destroy(f)


def test_identity_init(env):
    torch, abi, F = env
    f = abi.mem_flow_create(3)
    n = 4096
    u = torch.rand(n, D, dtype=torch.float32, device="cuda") * 0.98 + 0.01
    cond = torch.randn(C, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(u)
    lj = torch.zeros(n, dtype=torch.float32, device="cuda")
    abi.mem_flow_map(f, cond, u, y, lj)
    assert torch.max(torch.abs(y - u)).item() < 2e-6
    assert torch.max(torch.abs(lj)).item() < 1e-4
    abi.mem_destroy(f)


def test_random_flow_vs_reference(env):
    torch, abi, F = env
    layers = F.init_params(D, K, H, C, seed=5, zero_last=False)
    for L in layers:           # the GPU multiplies BF16 copies of W2 and W3
        L["W2"] = bf16(torch, L["W2"])
        L["W3"] = bf16(torch, L["W3"])
    f = abi.mem_flow_create(0)
    abi.mem_flow_set_params(f, F.to_flat(layers))
    rng = np.random.default_rng(6)
    n = 2048
    u = rng.uniform(0.02, 0.98, (n, D))
    c = rng.normal(size=C)
    yr, ljr = F.forward(layers, u, np.tile(c, (n, 1)))
    ug = torch.tensor(u, dtype=torch.float32, device="cuda")
    y = torch.zeros_like(ug)
    lj = torch.zeros(n, dtype=torch.float32, device="cuda")
    abi.mem_flow_map(f, torch.tensor(c, dtype=torch.float32, device="cuda"), ug, y, lj)
    dy = np.abs(y.cpu().numpy() - yr)
    dl = np.abs(lj.cpu().numpy() - ljr)
    assert np.median(dy) < 2e-3 and dy.max() < 5e-2, (np.median(dy), dy.max())
    assert np.median(dl) < 2e-2 and dl.max() < 2e-1, (np.median(dl), dl.max())
    abi.mem_destroy(f)


def test_density_normalised_on_gpu(env):
    torch, abi, F = env
    layers = F.init_params(D, K, H, C, seed=8, zero_last=False)
    f = abi.mem_flow_create(0)
    abi.mem_flow_set_params(f, F.to_flat(layers))
    n = 1 << 20
    g = torch.Generator(device="cuda").manual_seed(11)
    u = torch.rand(n, D, dtype=torch.float32, device="cuda", generator=g).clamp(1e-6, 1 - 1e-6)
    cond = torch.randn(C, dtype=torch.float32, device="cuda", generator=g)
    y = torch.zeros_like(u)
    lj = torch.zeros(n, dtype=torch.float32, device="cuda")
    abi.mem_flow_map(f, cond, u, y, lj)
    J = torch.exp(lj.double())
    mean, sd = J.mean().item(), J.std().item()
    assert abs(mean - 1.0) < 5 * sd / np.sqrt(n), (mean, sd)
    assert sd > 0.05   # the random flow is far from the identity
    abi.mem_destroy(f)


def _train_data(rng, n_items):
    """Samples concentrated around an item-dependent point (a learnable target)."""
    ys = np.empty((n_items, 128, D))
    cs = rng.normal(size=(n_items, C))
    for i in range(n_items):
        mu = 1 / (1 + np.exp(-0.8 * cs[i, :D]))
        ys[i] = np.clip(mu + 0.08 * rng.normal(size=(128, D)), 0.01, 0.99)
    ws = rng.uniform(0.5, 1.5, (n_items, 128))
    ws /= ws.sum(axis=1, keepdims=True)
    return ys, ws, cs


def test_gradients_vs_fp64_backprop(env):
    torch, abi, F = env
    rng = np.random.default_rng(21)
    layers = F.init_params(D, K, H, C, seed=9, zero_last=False)
    for L in layers:
        L["W2"] = bf16(torch, L["W2"])
        L["W3"] = bf16(torch, L["W3"])
    n_items = 6
    ys, ws, cs = _train_data(rng, n_items)
    f = abi.mem_flow_create(0)
    abi.mem_flow_set_params(f, F.to_flat(layers))
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda").contiguous()
    g_gpu, loss_gpu = abi.mem_flow_grad(f, t(ys), t(ws), t(cs))
    G = None
    loss_ref = 0.0
    for i in range(n_items):
        ci = np.tile(cs[i], (128, 1))
        Gi = F.grad(layers, ys[i], ws[i], ci)
        loss_ref += F.loss(layers, ys[i], ws[i], ci)
        G = Gi if G is None else [{k: G[l][k] + Gi[l][k] for k in G[l]} for l in range(K)]
    g_ref = F.to_flat(G)
    assert loss_gpu == pytest.approx(loss_ref, rel=2e-2, abs=2e-2)
    # the same backpropagation in FP64 with the GPU's BF16 operands: every operand
    # of the tensor-core products (hidden activations, W2, W3, dL/d(out), dL/da2)
    # rounded to BF16 as the kernels round it, accumulation exact
    rnd = lambda a: bf16(torch, a)
    Gr, loss_r = None, 0.0
    for i in range(n_items):
        ci = np.tile(cs[i], (128, 1))
        Gi = F.grad(layers, ys[i], ws[i], ci, rnd=rnd)
        loss_r += F.loss(layers, ys[i], ws[i], ci, rnd=rnd)
        Gr = Gi if Gr is None else [{k: Gr[l][k] + Gi[l][k] for k in Gr[l]} for l in range(K)]
    g_rnd = F.to_flat(Gr)
    assert loss_gpu == pytest.approx(loss_r, rel=1e-4, abs=1e-4)
    off = 0
    for l in range(K):
        for name in F.PARAM_ORDER:
            n = G[l][name].size
            a = g_gpu[off:off + n].astype(np.float64)
            b, br = g_ref[off:off + n], g_rnd[off:off + n]
            off += n
            nb = np.linalg.norm(b)
            if nb < 1e-9:
                continue
            # against the same BF16 operands: per tensor within 1e-3
            assert np.linalg.norm(a - br) / np.linalg.norm(br) < 1e-3, \
                (l, name, np.linalg.norm(a - br) / np.linalg.norm(br))
            # against exact arithmetic: the BF16 operands only perturb it
            cos = a @ b / (np.linalg.norm(a) * nb)
            assert cos > 0.98, (l, name, cos)
    abi.mem_destroy(f)


def test_training_lowers_loss(env):
    torch, abi, F = env
    rng = np.random.default_rng(22)
    ys, ws, cs = _train_data(rng, 256)
    t = lambda a: torch.tensor(a, dtype=torch.float32, device="cuda").contiguous()
    f = abi.mem_flow_create(1)
    trace = abi.mem_flow_train(f, t(ys), t(ws), t(cs), n_steps=300, batch_items=32, lr=2e-3)
    first, last = trace[:20].mean(), trace[-20:].mean()
    assert np.all(np.isfinite(trace))
    # identity flow: loss = sum w (-log sig'(logit y)) > 0 ... the trained flow concentrates mass
    assert last < first - 0.5 * 32, (first, last)
    abi.mem_destroy(f)
