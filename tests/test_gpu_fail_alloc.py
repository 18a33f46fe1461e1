"""Error paths under device-memory exhaustion, injected on the host: for every device
allocation that a graph build + solve + phase makes, a fresh context is told to fail
exactly there (qh_debug_fail_alloc).  The call that meets it must return QH_ENOMEM,
and the same context, with the injection off, must then give results bit-identical
to those of a context that never failed.  No GPU fault is involved: the allocation
is refused before the CUDA allocator is called.
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


def _reads():
    return synth.batched_blocks(1004, n_blocks=3, n_min=40, n_max=200)


def _snps():
    return synth.region_reads(33, n_snps=200, region=80_000, n_reads=60, len_mean=9000,
                              len_sd=3000, flip_p=0.08, miss_p=0.0, qual=(7, 30))


CASES = {  # (fragments, mode, storage, precision, replicas, step kernel)
    "read-tiles-bf16-multistep": (_reads, "read", 1, 1, 128, "multistep-stream-tile"),
    "read-tiles-fp8": (_reads, "read", 1, 3, 64, None),
    "snp-csr-bf16-band-refine": (_snps, "snp", 2, 1, 128, "csr-band8"),
    "snp-tiles-fp32-refine": (_snps, "snp", 1, 0, 64, None),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_every_allocation_failure_returns_enomem_and_context_recovers(q, case):
    make, mode, storage, precision, R, kernel = CASES[case]
    fr = make()
    qmode = q.MODE_READ if mode == "read" else q.MODE_SNP

    def run(c):
        g = c.build_graph(fr, mode=qmode, storage=storage)
        sol = c.solve(g, replicas=R, steps=120, precision=precision, seed=3, refine_max=4,
                      step_kernel=kernel)
        hap1, _, bid = c.phase(g, sol, fr.n_snps)
        return sol.cuts().copy(), sol.spins(g.n_nodes).copy(), hap1.copy(), bid.copy()

    def same(a, b):
        return all(np.array_equal(u, v) for u, v in zip(a, b))

    ref = run(q.Context(0))
    failures = 0
    for k in range(400):
        c = q.Context(0)
        c.debug_fail_alloc(k)
        try:
            out = run(c)
        except q.QhError as e:
            assert e.status == q.QH_ENOMEM, str(e)
            failures += 1
            c.debug_fail_alloc(-1)
            assert same(run(c), ref), (case, k)  # the context survives the failure
            continue
        assert same(out, ref)  # past the last allocation: nothing failed
        break
    else:
        pytest.fail("the path never completed")
    assert failures >= 20, failures  # each of the path's allocations failed once


def test_fail_alloc_argument_checked(q):
    c = q.Context(0)
    with pytest.raises(q.QhError):
        c.debug_fail_alloc(-2)
    c.debug_fail_alloc(-1)
