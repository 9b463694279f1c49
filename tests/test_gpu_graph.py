"""Batch graphs (blast_graph_*): one blast_cl_batch call captured into a CUDA
graph and launched again with the same buffers.

Bars: a launch gives the bits of the direct call on the same inputs (FP64 and
the tensor-core path, uneven tracer counts and ell subsets); after the input
arrays are rewritten in place, the next launch gives the direct call's bits on
the new inputs; direct calls on the plan between launches (which may grow the
plan's own work space) do not disturb the graph; launches take no device
memory; host inputs are refused.
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

FIELDS = ["kern_chi", "kern_Rchi", "growth_chi", "growth_Rchi", "k_tab", "p_tab"]


def subset_request(full, ng, ns, max_clust):
    kc = np.concatenate([full.kern_chi[:ng], full.kern_chi[max_clust:max_clust + ns]])
    kR = np.concatenate([full.kern_Rchi[:ng], full.kern_Rchi[max_clust:max_clust + ns]])
    return synth.Request(ng, ns, np.ascontiguousarray(kc), np.ascontiguousarray(kR), full.growth_chi,
                         full.growth_Rchi, full.k_tab, full.p_tab)


@pytest.fixture(scope="module")
def tc_plan():
    p = bl.Plan(synth.plan_spec("tc"))
    p.precompute(bl.BASIS_ALL)
    yield p
    p.close()


def _batch(plan, seed0):
    spec = plan.spec
    chi, R, _ = plan.nodes()
    L = spec.ells.size
    shapes = [(spec.max_clust, spec.max_lens), (1, 1), (2, 0)]
    sels = [None, [0, L - 1], list(range(1, L, 2))]
    rqs = [subset_request(synth.config_request("tc", chi, R, seed0 + i), ng, ns, spec.max_clust)
           for i, (ng, ns) in enumerate(shapes)]
    return rqs, sels


def _direct(plan, rqs, sels, prec):
    import torch
    dev = [{f: torch.from_numpy(np.ascontiguousarray(getattr(rq, f))).cuda() for f in FIELDS} for rq in rqs]
    reqs = [plan.request(rq, ell_sel=s, device_arrays=d) for rq, s, d in zip(rqs, sels, dev)]
    outs = [torch.empty((bl.blast_npairs(rq.n_clust, rq.n_lens), plan.n_sel(s)), dtype=torch.float64, device="cuda")
            for rq, s in zip(rqs, sels)]
    s = torch.cuda.current_stream().cuda_stream
    assert bl.blast_cl_batch(plan.h, reqs, prec, [o.data_ptr() for o in outs], 1, s) == bl.BLAST_OK
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


@pytest.mark.parametrize("prec", [bl.BLAST_FP64, bl.BLAST_BF16S])
def test_graph_launches_equal_direct_calls(tc_plan, prec):
    import torch
    plan = tc_plan
    rqs, sels = _batch(plan, 400)
    dev = [{f: torch.from_numpy(np.ascontiguousarray(getattr(rq, f))).cuda() for f in FIELDS} for rq in rqs]
    reqs = [plan.request(rq, ell_sel=s, device_arrays=d) for rq, s, d in zip(rqs, sels, dev)]
    outs = [torch.full((bl.blast_npairs(rq.n_clust, rq.n_lens), plan.n_sel(s)), float("nan"), dtype=torch.float64,
                       device="cuda") for rq, s in zip(rqs, sels)]
    g = bl.blast_graph_create(plan.h, reqs, prec, [o.data_ptr() for o in outs])
    try:
        assert bl.blast_graph_reserved(g) > 0
        stream = torch.cuda.current_stream().cuda_stream
        assert bl.blast_graph_launch(g, stream) == bl.BLAST_OK
        torch.cuda.synchronize()
        ref = _direct(plan, rqs, sels, prec)
        for o, r in zip(outs, ref):
            assert np.array_equal(o.cpu().numpy(), r)
        # new cosmologies written into the same device arrays
        rqs2, _ = _batch(plan, 500)
        for d, rq in zip(dev, rqs2):
            for f in FIELDS:
                d[f].copy_(torch.from_numpy(np.ascontiguousarray(getattr(rq, f))))
        # a direct call with a larger batch in between grows the plan's own work space
        big, bsel = _batch(plan, 600)
        _direct(plan, big * 3, bsel * 3, prec)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            assert bl.blast_graph_launch(g, stream) == bl.BLAST_OK
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        ref2 = _direct(plan, rqs2, sels, prec)
        for o, r, r1 in zip(outs, ref2, ref):
            assert np.array_equal(o.cpu().numpy(), r)
            assert not np.array_equal(r, r1)
    finally:
        bl.blast_graph_destroy(g)


def test_graph_refuses_host_inputs(tc_plan):
    import torch
    plan = tc_plan
    rqs, sels = _batch(plan, 700)
    reqs = [plan.request(rq, ell_sel=s) for rq, s in zip(rqs, sels)]  # host arrays
    outs = [torch.empty((bl.blast_npairs(rq.n_clust, rq.n_lens), plan.n_sel(s)), dtype=torch.float64, device="cuda")
            for rq, s in zip(rqs, sels)]
    with pytest.raises(bl.BlastError) as ei:
        bl.blast_graph_create(plan.h, reqs, bl.BLAST_BF16S, [o.data_ptr() for o in outs])
    assert ei.value.status == bl.BLAST_EINVAL
