"""The bounded device waits of the tensor-core contraction, made to run out.

A test hook has one epilogue warp of the first CTA wait on a barrier that
nothing completes, with a short limit.  The wait gives up, the kernel records
its error word and every warp leaves once its copies and MMAs in flight are
done; the call returns BLAST_ETIMEOUT.  Nothing faults or hangs, and the next
call on the same plan and context gives the same C_l as before.
"""
import numpy as np
import pytest

from paper_2410_03632_gb300 import blast as bl
from paper_2410_03632_gb300 import synth

pytestmark = pytest.mark.gpu


def _have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


if not _have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_bounded_wait_runs_out_and_the_context_survives():
    spec = synth.plan_spec("tc")
    plan = bl.Plan(spec)
    try:
        plan.precompute(bl.BASIS_ALL)
        chi, R, _ = plan.nodes()
        rqs = [synth.config_request("tc", chi, R, i) for i in range(4)]
        ref = plan.cl_batch(rqs, bl.BLAST_BF16S)
        assert bl.blast_test_trip_wait(plan.h, 5) == bl.BLAST_OK
        with pytest.raises(bl.BlastError) as ei:
            plan.cl_batch(rqs, bl.BLAST_BF16S)
        assert ei.value.status == bl.BLAST_ETIMEOUT
        again = plan.cl_batch(rqs, bl.BLAST_BF16S)
        for a, b in zip(again, ref):
            assert np.array_equal(a, b)
        assert bl.blast_test_trip_wait(plan.h, -2) == bl.BLAST_EINVAL
    finally:
        plan.close()
