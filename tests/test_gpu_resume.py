"""Resume from a saved state: steps t0 .. t0+2n run in one call and as two calls of n
steps (the state x, y copied out and back in between, as a checkpoint would) give
bit-identical states, on every step-kernel family.  The product operand is not part
of the saved state: every kernel rebuilds it from x exactly as its epilogue writes it.
"""
import numpy as np
import pytest

from paper_2603_25762_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_25762_gb300 import build, qhap
    build.build()
    return qhap


@pytest.fixture(scope="module")
def ctx(q):
    return q.Context(0)


CASES = [  # (precision, step kernel, storage, R, SB variant)
    (0, None, 1, 64, "ballistic"),
    (1, "cta-bn128-s2-x3", 1, 128, "ballistic"),
    (1, "persistent-bn64-tma-state", 1, 128, "discrete"),
    (1, "multistep-stream-tile", 1, 256, "ballistic"),
    (1, "multistep-jres-group", 1, 256, "adiabatic"),
    (3, None, 1, 128, "ballistic"),
    (0, "csr-lane8", 2, 64, "discrete"),
    (1, "csr-lane8", 2, 128, "ballistic"),
    (1, "csr-band8", 2, 128, "ballistic"),
]


@pytest.mark.parametrize("precision,kernel,storage,R,variant", CASES)
def test_split_step_range_is_bit_identical(q, ctx, precision, kernel, storage, R, variant):
    import torch
    fr = synth.batched_blocks(1004, n_blocks=4, n_min=80, n_max=300)
    g = ctx.build_graph(fr, mode=q.MODE_READ, storage=storage)
    n_pad, pidx, c0 = g.layout()
    rng = np.random.default_rng(9)
    x = np.zeros((R, n_pad), np.float32)
    y = np.zeros((R, n_pad), np.float32)
    real = pidx[pidx >= 0]
    x[:, real] = rng.uniform(-0.1, 0.1, (R, real.size))
    y[:, real] = rng.uniform(-0.1, 0.1, (R, real.size))
    dt = 0.25 if variant == "adiabatic" else 1.0  # aSB diverges at 0.5 from mid-schedule
    t0, n, steps = 101, 20, 400  # an odd t0: the operand's double buffer starts on its odd side
    kw = dict(dt=dt, c0=c0, step_kernel=kernel, variant=variant)
    xa, ya = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ctx.debug_steps(g, precision, R, xa, ya, t0, 2 * n, steps, **kw)
    xb, yb = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ctx.debug_steps(g, precision, R, xb, yb, t0, n, steps, **kw)
    saved = (xb.cpu().numpy().copy(), yb.cpu().numpy().copy())  # the checkpoint
    xc, yc = torch.from_numpy(saved[0]).cuda(), torch.from_numpy(saved[1]).cuda()
    ctx.debug_steps(g, precision, R, xc, yc, t0 + n, n, steps, **kw)
    assert not np.array_equal(saved[0], x)  # the steps moved the state
    assert np.isfinite(xa.cpu().numpy()).all() and np.isfinite(ya.cpu().numpy()).all()
    assert np.array_equal(xc.cpu().numpy(), xa.cpu().numpy())
    assert np.array_equal(yc.cpu().numpy(), ya.cpu().numpy())
