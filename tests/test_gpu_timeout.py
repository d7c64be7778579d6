"""The bounded-wait path: a device wait that cannot complete gives RLOBPCG_ERR_TIMEOUT, releases
the TMEM its kernel held, and leaves the stream and the GPU usable.

rlobpcg_check_bounded_wait runs a kernel that allocates TMEM and waits, with a short bound, on an
mbarrier that nothing arrives at or on a global flag that nothing sets -- the primitives every
wait of the tensor-core Gram kernels and of the dataflow QR uses. After it, a split Gram pass
(which allocates all 512 TMEM columns of its SM) and a whole solve must still give the oracle's
results: a leaked TMEM allocation or a broken context would fail them.
"""
import numpy as np
import pytest

import oracle
from paper_2602_16797_gb300 import rlobpcg as rl
from paper_2602_16797_gb300 import workloads as wl
from tests.parity import check_sigma

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [0, 1])
def test_wait_that_cannot_complete_times_out_and_releases(kind):
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(3):
        assert rl.rlobpcg_check_bounded_wait(kind, 1000, st) == rl.RLOBPCG_ERR_TIMEOUT
        assert "bounded device wait ran out" in rl.rlobpcg_last_error()
    assert rl.rlobpcg_check_bounded_wait(kind, 0, st) == rl.RLOBPCG_ERR_INVALID_ARG
    assert rl.rlobpcg_check_bounded_wait(2, 10, st) == rl.RLOBPCG_ERR_INVALID_ARG
    # the GPU still runs the tensor-core Gram pass (all of TMEM) and a whole solve correctly
    from tests.test_gpu_split_gram import check_against_oracle
    rng = np.random.default_rng(8)
    check_against_oracle(rng.standard_normal((3000, 300)), rng.standard_normal((300, 5)))
    A, s, V = wl.planted_small_gap_free()
    o = rl.rlobpcg_default_opts()
    o.seed = 4
    o.fixed_iters = 5
    sig, Vg, _, _, info = rl.solve(torch.from_numpy(A).cuda(), 1, opts=o)
    ref = oracle.rlobpcg(A, k=1, seed=4, fixed_iters=5)
    check_sigma(sig.cpu().numpy(), ref["sigma"], ref["sigma11"], 50)
