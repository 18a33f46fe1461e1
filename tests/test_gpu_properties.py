"""Symmetries that hold bit for bit on the GPU, independently of the oracle:

- spin flip: the SB step is odd in (x, y), so a run from (-x, -y) ends at exactly minus
  the run from (x, y);
- gauge: negating the alleles of a set S of reads gives the read graph D W D (d = -1 on
  S), and a run on it from (D x, D y) ends at exactly D times the run on W.

Both rest on every kernel summing in a fixed order and rounding symmetrically: a row's
product terms all change sign together, so does their sum, and the update, the wall,
sgn and the cubic term are odd.  Initial values are never exactly zero (sgn(0) = +1
is the one asymmetric point).
"""
import dataclasses

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
    (1, "multistep-stream-tile", 1, 256, "discrete"),
    (1, "multistep-jres-group", 1, 256, "ballistic"),
    (3, None, 1, 128, "ballistic"),
    (0, "csr-lane8", 2, 64, "adiabatic"),
    (1, "csr-band8", 2, 128, "ballistic"),
]


def _state(n_pad, pidx, R, seed):
    rng = np.random.default_rng(seed)
    x = np.zeros((R, n_pad), np.float32)
    y = np.zeros((R, n_pad), np.float32)
    real = pidx[pidx >= 0]
    sgn = np.where(rng.random((R, real.size)) < 0.5, -1.0, 1.0)
    x[:, real] = sgn * rng.uniform(0.01, 0.1, (R, real.size))  # never exactly zero
    y[:, real] = rng.uniform(-0.1, 0.1, (R, real.size))
    return x, y


def _run(q, ctx, g, precision, R, x, y, kernel, variant):
    import torch
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    _, _, c0 = g.layout()
    dt = 0.25 if variant == "adiabatic" else 1.0
    ctx.debug_steps(g, precision, R, xd, yd, 101, 12, 400, dt=dt, c0=c0, step_kernel=kernel,
                    variant=variant)
    return xd.cpu().numpy(), yd.cpu().numpy()


def _exact(a, b, what):
    assert np.isfinite(a).all()
    assert np.array_equal(a, b), f"{what}: max |diff| {np.abs(a - b).max():.3g}"


@pytest.mark.parametrize("precision,kernel,storage,R,variant", CASES)
def test_spin_flip_symmetry_bit_exact(q, ctx, precision, kernel, storage, R, variant):
    fr = synth.batched_blocks(1004, n_blocks=4, n_min=80, n_max=300)
    g = ctx.build_graph(fr, mode=q.MODE_READ, storage=storage)
    n_pad, pidx, _ = g.layout()
    x, y = _state(n_pad, pidx, R, 3)
    x1, y1 = _run(q, ctx, g, precision, R, x, y, kernel, variant)
    x2, y2 = _run(q, ctx, g, precision, R, -x, -y, kernel, variant)
    assert not np.array_equal(x1, x)
    _exact(x2, -x1, "x")
    _exact(y2, -y1, "y")


@pytest.mark.parametrize("precision,kernel,storage,R,variant", CASES)
def test_gauge_invariance_bit_exact(q, ctx, precision, kernel, storage, R, variant):
    fr = synth.batched_blocks(1004, n_blocks=4, n_min=80, n_max=300)
    rng = np.random.default_rng(8)
    flip = rng.random(fr.n_frags) < 0.5  # the reads of S
    per_entry = np.repeat(flip, np.diff(fr.frag_ptr))
    frd = dataclasses.replace(fr, allele=np.where(per_entry, -fr.allele, fr.allele).astype(fr.allele.dtype))
    g = ctx.build_graph(fr, mode=q.MODE_READ, storage=storage)
    gd = ctx.build_graph(frd, mode=q.MODE_READ, storage=storage)
    n_pad, pidx, c0 = g.layout()
    n_pad_d, pidx_d, c0_d = gd.layout()
    assert n_pad_d == n_pad and np.array_equal(pidx_d, pidx) and np.array_equal(c0_d, c0)
    d = np.ones(n_pad, np.float32)
    d[pidx[flip & (pidx >= 0)]] = -1.0
    x, y = _state(n_pad, pidx, R, 4)
    x1, y1 = _run(q, ctx, g, precision, R, x, y, kernel, variant)
    x2, y2 = _run(q, ctx, gd, precision, R, x * d, y * d, kernel, variant)
    _exact(x2, x1 * d, "x")
    _exact(y2, y1 * d, "y")
