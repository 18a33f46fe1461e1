"""qh_matvec_bf16_noalloc: the BF16 J x X product for callers that are not free to
allocate GPU memory -- a host whose own allocator already owns the device memory (an
extra cudaMalloc would fail or escape its accounting), or a process held to a fixed
device-memory budget.

It must give the same Z as the allocating entry point qh_debug_matvec(BF16) on calls
in a row (the shared static scratch keeps the previous call's contents, which must
not leak into the next result), make no device allocation at all (checked with the
library's allocation-failure hook armed), and reject sizes beyond its fixed array.
This file is collected last so that a stop at the first failure has run every other
test before it.
"""
import numpy as np
import pytest

from paper_2603_25762_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel_frob(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def q():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_25762_gb300 import build, qhap
    build.build()
    return qhap


def _state(n_pad, pidx, R, seed):
    import torch
    rng = np.random.default_rng(seed)
    x = np.zeros((R, n_pad), np.float32)
    inb = pidx >= 0
    x[:, pidx[inb]] = rng.uniform(-1, 1, size=(R, int(inb.sum())))
    return torch.from_numpy(x).cuda()


def _same(zn, zr, what):
    assert np.isfinite(zn).all(), what
    # same operands, same kernel: within the BF16 path's 1e-2 bar, and in fact equal
    assert _rel_frob(zn.astype(np.float64), zr.astype(np.float64)) <= 1e-2, what
    assert np.array_equal(zn, zr), what


def test_noalloc_matches_allocating_matvec_twice(q):
    import torch
    ctx = q.Context(0)
    fr = synth.hifi_region(1002, scale=0.08)
    g = ctx.build_graph(fr)
    n_pad, pidx, _ = g.layout()
    R = 128
    for call in range(2):
        xd = _state(n_pad, pidx, R, 12 + call)
        z_ref = torch.zeros_like(xd)
        ctx.debug_matvec(g, q.PREC_BF16, R, xd, z_ref)
        z = torch.full_like(xd, float("nan"))  # stale output must be overwritten
        ctx.matvec_bf16_noalloc(g, R, xd, z)
        _same(z.cpu().numpy(), z_ref.cpu().numpy(), f"call {call}")


def test_noalloc_makes_no_allocation_and_keeps_no_state_between_calls(q):
    """Reference products first (allocating entry point, own context).  Then a fresh
    context whose every further device allocation fails: the allocating entry point
    fails there with QH_ENOMEM, while the no-allocation entry point serves a sequence
    of calls -- replica counts 192 (64-replica tiles), 64, a larger graph, then a
    smaller graph -- each equal to its reference."""
    import torch
    ref_ctx = q.Context(0)
    frs = [synth.hifi_region(1002, scale=0.08), synth.batched_blocks(1004, n_blocks=5,
                                                                       n_min=40, n_max=300)]
    calls = [(0, 192, 31), (0, 64, 32), (1, 256, 33), (0, 128, 34), (1, 64, 35)]
    refs = []
    for gi, R, seed in calls:
        g = ref_ctx.build_graph(frs[gi])
        n_pad, pidx, _ = g.layout()
        xd = _state(n_pad, pidx, R, seed)
        z = torch.zeros_like(xd)
        ref_ctx.debug_matvec(g, q.PREC_BF16, R, xd, z)
        refs.append((xd, z.cpu().numpy()))
    ctx = q.Context(0)
    graphs = [ctx.build_graph(fr) for fr in frs]
    ctx.debug_fail_alloc(0)  # every later device allocation of this context fails
    try:
        xd0, _ = refs[0]
        with pytest.raises(q.QhError) as e:
            ctx.debug_matvec(graphs[0], q.PREC_BF16, 192, xd0, torch.zeros_like(xd0))
        assert e.value.status == q.QH_ENOMEM
        for (gi, R, _), (xd, zr) in zip(calls, refs):
            z = torch.full_like(xd, float("nan"))
            ctx.matvec_bf16_noalloc(graphs[gi], R, xd, z)
            _same(z.cpu().numpy(), zr, f"graph {gi}, R = {R}")
    finally:
        ctx.debug_fail_alloc(-1)


def test_noalloc_rejects_sizes_beyond_the_static_array(q):
    import torch
    ctx = q.Context(0)
    g = ctx.build_graph(synth.hifi_region(1002, scale=0.08))
    n_pad, _, _ = g.layout()
    R = 64 * ((4_194_304 // n_pad) // 64 + 1)  # first multiple of 64 past the limit
    x = torch.zeros(R * n_pad, dtype=torch.float32, device="cuda")
    z = torch.zeros_like(x)
    with pytest.raises(q.QhError) as e:
        ctx.matvec_bf16_noalloc(g, R, x, z)
    assert e.value.status == q.QH_EINVAL
    assert "4,194,304" in str(e.value)
    with pytest.raises(q.QhError):
        ctx.matvec_bf16_noalloc(g, 96, x, z)  # not a multiple of 64
