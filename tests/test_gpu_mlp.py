"""Surrogate MLP kernels (through the C ABI) against the FP64 oracle MLP.  GPU.

The oracle is run with the bfloat16-rounded weights the kernels read, so the
remaining difference is FP32 vs FP64 arithmetic."""
import ctypes as C

import numpy as np
import pytest

from oracle import mlp_oracle as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_07083_gb300 import build as B
    B.build()
    from paper_2605_07083_gb300 import pic
    return torch, pic, pic.load()


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _bf16_theta(theta32):
    """The parameters the kernels use: bfloat16 weights, FP32 biases."""
    th = np.asarray(theta32, np.float64).copy()
    p = 0
    for i, o in zip(M.SIZES[:-1], M.SIZES[1:]):
        th[p:p + o * i] = M.bf16_round(theta32[p:p + o * i])
        p += o * i + o
    return th


def _setup(torch, lib, seed, batch):
    rng = np.random.default_rng(seed)
    theta = (rng.standard_normal(M.param_count()) * 0.15).astype(np.float32)
    x = rng.standard_normal((batch, 5)).astype(np.float32)
    t = rng.standard_normal((batch, 4)).astype(np.float32)
    master = torch.from_numpy(theta).cuda()
    w = torch.empty(M.param_count(), dtype=torch.int16, device="cuda")
    assert lib.pic_mlp_cast_bf16(_ptr(master), _ptr(w), None) == 0
    return theta, x, t, master, w


@pytest.mark.parametrize("batch", [1, 100, 4096])
def test_forward_matches_oracle(env, batch):
    torch, pic, lib = env
    theta, x, t, master, w = _setup(torch, lib, 1, batch)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty((batch, 4), dtype=torch.float32, device="cuda")
    assert lib.pic_mlp_forward(_ptr(master), _ptr(w), _ptr(xd), batch, _ptr(y), None) == 0
    torch.cuda.synchronize()
    yo, _ = M.forward(_bf16_theta(theta), x.astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), yo, rtol=1e-4, atol=1e-5 * np.abs(yo).max())


@pytest.mark.parametrize("batch", [37, 4096])
def test_gradient_matches_oracle(env, batch):
    torch, pic, lib = env
    theta, x, t, master, w = _setup(torch, lib, 2, batch)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    nbytes = lib.pic_mlp_scratch_bytes(batch)
    scratch = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    g = torch.empty(M.param_count(), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    rc = lib.pic_mlp_grad(_ptr(master), _ptr(w), _ptr(xd), _ptr(td), batch, _ptr(g), _ptr(loss),
                          _ptr(scratch), nbytes, None)
    assert rc == 0
    torch.cuda.synchronize()
    Lo, go = M.loss_and_grad(_bf16_theta(theta), x.astype(np.float64), t.astype(np.float64))
    assert loss.item() == pytest.approx(Lo, rel=1e-5)
    gg = g.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(gg, go, rtol=1e-3, atol=1e-5 * np.abs(go).max())
    # deterministic: a second evaluation is bit-identical
    g2 = torch.empty_like(g)
    lib.pic_mlp_grad(_ptr(master), _ptr(w), _ptr(xd), _ptr(td), batch, _ptr(g2), None,
                     _ptr(scratch), nbytes, None)
    assert torch.equal(g, g2)


def test_adam_step_matches_oracle_and_training_converges(env):
    torch, pic, lib = env
    batch = 512
    theta, x, _, master, w = _setup(torch, lib, 3, batch)
    t = np.stack([np.tanh(x[:, 0]), 0.5 * x[:, 1], np.sin(x[:, 2]), 0.1 * x[:, 3] * x[:, 4]],
                 1).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    m = torch.zeros(M.param_count(), device="cuda")
    v = torch.zeros(M.param_count(), device="cuda")
    nbytes = lib.pic_mlp_scratch_bytes(batch)
    scratch = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    lr, b1, b2, eps = 1e-3, 0.9, 0.999, 1e-8
    # one step against the oracle's Adam on the oracle's gradient
    Lo, go = M.loss_and_grad(_bf16_theta(theta), x.astype(np.float64), t.astype(np.float64))
    rc = lib.pic_mlp_train_step(_ptr(master), _ptr(w), _ptr(m), _ptr(v), 1, lr, b1, b2, eps,
                                _ptr(xd), _ptr(td), batch, _ptr(loss), _ptr(scratch), nbytes, None)
    assert rc == 0
    torch.cuda.synchronize()
    th_o, _, _ = M.adam_step(theta.astype(np.float64), go, np.zeros_like(go), np.zeros_like(go), 1,
                             lr, b1, b2, eps)
    d_gpu = master.cpu().numpy().astype(np.float64) - theta
    d_ora = th_o - theta
    close = np.abs(d_gpu - d_ora) <= 1e-3 * lr + 1e-3 * np.abs(d_ora)
    # an update is +-lr unless |g| is near eps: only near-zero gradients may differ
    assert (~close).sum() <= 0.002 * close.size
    assert np.all(np.abs(go[~close]) < 1e-6)
    # the bfloat16 copy is the round-to-nearest-even of the updated master
    wb = (w.cpu().numpy().view(np.uint16).astype(np.uint32) << 16).view(np.float32)
    np.testing.assert_array_equal(wb.astype(np.float64), M.bf16_round(master.cpu().numpy()))
    first = loss.item()
    for k in range(2, 301):
        lib.pic_mlp_train_step(_ptr(master), _ptr(w), _ptr(m), _ptr(v), k, 3e-3, b1, b2, eps,
                               _ptr(xd), _ptr(td), batch, _ptr(loss), _ptr(scratch), nbytes, None)
    torch.cuda.synchronize()
    assert loss.item() < 0.2 * first
