"""blast_cl_noalloc: FP64 C_l without any device allocation.

Some callers cannot allocate device memory while they evaluate: a host
framework that has reserved the GPU's memory for its own pool allocator (a
cudaMalloc behind its back can fail or fragment that pool), or a
latency-critical request loop where cudaMalloc / cudaFree would synchronise the
device.  For them the library takes the evaluation's scratch from a fixed
device array compiled into it.  These tests call that entry point through the
C ABI and compare it with blast_cl's FP64 result, on consecutive calls that
reuse the same array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2410_03632_gb300 import blast as bl
from paper_2410_03632_gb300 import synth
from tests.metrics import eij

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def _torch_cuda():
    try:
        import torch
        return torch if torch.cuda.is_available() else None
    except Exception:
        return None


torch = _torch_cuda()
if torch is None:
    pytest.skip("needs a CUDA device", allow_module_level=True)

FIELDS = ["kern_chi", "kern_Rchi", "growth_chi", "growth_Rchi", "k_tab", "p_tab"]


def to_device(rq):
    return {f: torch.from_numpy(np.ascontiguousarray(getattr(rq, f))).cuda() for f in FIELDS}


@pytest.fixture(scope="module")
def small_plan():
    spec = synth.plan_spec("small")
    plan = bl.Plan(spec)
    plan.precompute(bl.BLAST_BASIS_FP64)
    yield spec, plan
    plan.close()


def test_noalloc_matches_blast_cl_on_consecutive_calls(small_plan):
    spec, plan = small_plan
    chi, R, _ = plan.nodes()
    stream = torch.cuda.current_stream().cuda_stream
    L = spec.ells.size
    cases = [(0, None), (1, None), (1, [0, 3, L - 1])]  # two full calls in a row, then a subset
    for idx, sel in cases:
        rq = synth.config_request("small", chi, R, idx)
        dev = to_device(rq)
        r = plan.request(rq, ell_sel=sel, device_arrays=dev)
        n_sel = L if sel is None else len(sel)
        out = torch.full((bl.blast_npairs(rq.n_clust, rq.n_lens), n_sel), float("nan"),
                         dtype=torch.float64, device="cuda")
        rc = bl.blast_cl_noalloc(plan.h, r, out.data_ptr(), stream)
        assert rc == bl.BLAST_OK, bl.blast_status_str(rc)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = plan.cl(rq, bl.BLAST_FP64, ell_sel=sel)
        assert np.all(np.isfinite(got))
        assert np.max(eij(got, ref, rq.n_clust, rq.n_lens)) < TOL_FP64


def test_noalloc_takes_no_device_memory(small_plan):
    """After plan creation (which places the fixed array and the kernels' code on
    the device) a call changes neither the driver's free-memory count nor the
    plan's work space: the evaluation's scratch is the fixed array."""
    spec, plan = small_plan
    chi, R, _ = plan.nodes()
    stream = torch.cuda.current_stream().cuda_stream
    P = None
    outs, devs = [], []
    for idx in (3, 4):
        rq = synth.config_request("small", chi, R, idx)
        devs.append((rq, to_device(rq)))
        P = bl.blast_npairs(rq.n_clust, rq.n_lens)
        outs.append(torch.empty((P, spec.ells.size), dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for (rq, dev), out in zip(devs, outs):
        r = plan.request(rq, device_arrays=dev)
        assert bl.blast_cl_noalloc(plan.h, r, out.data_ptr(), stream) == bl.BLAST_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    for (rq, _), out in zip(devs, outs):
        ref = plan.cl(rq, bl.BLAST_FP64)
        assert np.max(eij(out.cpu().numpy(), ref, rq.n_clust, rq.n_lens)) < TOL_FP64


def test_noalloc_refuses_what_blast_cl_refuses(small_plan):
    """Misaligned pointers and ell-mask bits beyond the plan are refused before
    anything is launched, as blast_cl refuses them."""
    spec, plan = small_plan
    chi, R, _ = plan.nodes()
    rq = synth.config_request("small", chi, R, 0)
    dev = to_device(rq)
    P = bl.blast_npairs(rq.n_clust, rq.n_lens)
    out = torch.full((P * spec.ells.size + 1,), 7.0, dtype=torch.float64, device="cuda")
    r = plan.request(rq, device_arrays=dev)
    r.ell_mask_lo = 1 << spec.ells.size      # one bit past the plan's last ell
    assert bl.blast_cl_noalloc(plan.h, r, out.data_ptr(), None) == bl.BLAST_EINVAL
    r = plan.request(rq, device_arrays=dev)
    assert bl.blast_cl_noalloc(plan.h, r, out.data_ptr() + 4, None) == bl.BLAST_EINVAL
    r.kern_Rchi = r.kern_Rchi + 4
    assert bl.blast_cl_noalloc(plan.h, r, out.data_ptr(), None) == bl.BLAST_EINVAL
    torch.cuda.synchronize()
    assert bool(torch.all(out == 7.0))      # nothing was written


def test_noalloc_rejects_host_inputs_and_oversized_requests(small_plan):
    spec, plan = small_plan
    chi, R, _ = plan.nodes()
    rq = synth.config_request("small", chi, R, 0)
    host_req = plan.request(rq)  # mem_space 0
    out = torch.empty((bl.blast_npairs(rq.n_clust, rq.n_lens), spec.ells.size), dtype=torch.float64,
                      device="cuda")
    assert bl.blast_cl_noalloc(plan.h, host_req, out.data_ptr(), None) == bl.BLAST_EINVAL
    # a grid whose per-request scratch exceeds the fixed array is refused before any device work
    big = synth.plan_spec("small")
    big.n_chi, big.n_R, big.max_clust, big.max_lens = 401, 256, 16, 16
    bp = bl.Plan(big)
    n = big.n_chi * big.n_R
    fake = {f: torch.zeros(max(n * 32, 1024), dtype=torch.float64, device="cuda") for f in FIELDS}
    req = bl.blast_request()
    req.n_clust, req.n_lens, req.n_ptab, req.mem_space = 16, 16, 256, 1
    for f in FIELDS:
        setattr(req, f, fake[f].data_ptr())
    assert bl.blast_cl_noalloc(bp.h, req, out.data_ptr(), None) == bl.BLAST_ENOMEM
    bp.close()
