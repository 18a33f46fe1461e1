"""qh_matvec_bf16_noalloc: the BF16 J x X product for callers that cannot allocate
device memory (for example code running during CUDA graph capture, host callbacks,
or hosts that hand out GPU memory through their own allocator).

It must give the same Z as the allocating entry point qh_debug_matvec(BF16) on two
calls in a row (the shared static scratch keeps the previous call's contents, which
must not leak into the next result), and reject sizes beyond its fixed array.
This file is collected last so that a stop at the first failure has run every other
test before it.
"""
import numpy as np
import pytest

from paper_2603_25762_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel_frob(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_noalloc_matches_allocating_matvec_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_25762_gb300 import build, qhap
    build.build()
    ctx = qhap.Context(0)
    fr = synth.hifi_region(1002, scale=0.08)
    g = ctx.build_graph(fr)
    n_pad, pidx, _ = g.layout()
    R = 128
    rng = np.random.default_rng(12)
    for call in range(2):
        x = np.zeros((R, n_pad), np.float32)
        inb = pidx >= 0
        x[:, pidx[inb]] = rng.uniform(-1, 1, size=(R, int(inb.sum())))
        xd = torch.from_numpy(x).cuda()
        z_ref = torch.zeros_like(xd)
        ctx.debug_matvec(g, qhap.PREC_BF16, R, xd, z_ref)
        z = torch.full_like(xd, float("nan"))  # stale output must be overwritten
        ctx.matvec_bf16_noalloc(g, R, xd, z)
        zr, zn = z_ref.cpu().numpy(), z.cpu().numpy()
        assert np.isfinite(zn).all(), f"call {call}"
        # same operands, same kernel: within the BF16 path's 1e-2 bar, and in fact equal
        assert _rel_frob(zn.astype(np.float64), zr.astype(np.float64)) <= 1e-2, f"call {call}"
        assert np.array_equal(zn, zr), f"call {call}"


def test_noalloc_rejects_sizes_beyond_the_static_array():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_25762_gb300 import build, qhap
    build.build()
    ctx = qhap.Context(0)
    g = ctx.build_graph(synth.hifi_region(1002, scale=0.08))
    n_pad, _, _ = g.layout()
    R = 64 * ((4_194_304 // n_pad) // 64 + 1)  # first multiple of 64 past the limit
    x = torch.zeros(R * n_pad, dtype=torch.float32, device="cuda")
    z = torch.zeros_like(x)
    with pytest.raises(qhap.QhError) as e:
        ctx.matvec_bf16_noalloc(g, R, x, z)
    assert e.value.status == qhap.QH_EINVAL
    assert "4,194,304" in str(e.value)
    with pytest.raises(qhap.QhError):
        ctx.matvec_bf16_noalloc(g, 96, x, z)  # not a multiple of 64
