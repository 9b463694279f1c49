"""The symmetrised chi-R form (App. A: R in (0, 1], both kernel orders) through
the C ABI against the oracle's symmetrised form.

Bars as for the split form: R nodes equal the oracle's; basis within 1e-11 of
its row maximum; FP64 C_l within e_ij <= 1e-10 and FP32 within 1e-4 of the
oracle for uneven tracer counts and ell subsets; the allocation-free entry
point gives blast_cl's FP64 bits; the non-separable entry refuses such plans
with BLAST_EINVAL.  On tensor-core shapes (one and two tracer groups) the
five-slice path is within e_ij <= 1e-4 of the oracle, and a cosmology's
result is the same alone and in a batch.
"""
import dataclasses

import numpy as np
import pytest

import oracle as orc
from paper_2410_03632_gb300 import blast as bl
from paper_2410_03632_gb300 import synth
from tests.metrics import eij

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_FP32 = 1e-4
TOL_BASIS = 1e-11


def _have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


if not _have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def subset_request(full, ng, ns, max_clust):
    kc = np.concatenate([full.kern_chi[:ng], full.kern_chi[max_clust:max_clust + ns]])
    kR = np.concatenate([full.kern_Rchi[:ng], full.kern_Rchi[max_clust:max_clust + ns]])
    return synth.Request(ng, ns, np.ascontiguousarray(kc), np.ascontiguousarray(kR), full.growth_chi,
                         full.growth_Rchi, full.k_tab, full.p_tab)


@pytest.fixture(scope="module", params=["tiny", "small"])
def case(request):
    spec = dataclasses.replace(synth.plan_spec(request.param), r_form=1)
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map, r_form=1)
    To = g.basis()
    plan = bl.Plan(spec)
    plan.precompute(bl.BASIS_ALL)
    yield request.param, spec, g, To, plan
    plan.close()


def _oracle(g, To, rq, sel=None):
    a = g.fit(rq.k_tab, rq.p_tab)
    T = To if sel is None else To[:, sel]
    return g.cl(T, a, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi,
                ell_subset=None if sel is None else g.ells[sel])


def test_nodes_and_basis(case):
    name, spec, g, To, plan = case
    chi, R, _ = plan.nodes()
    assert np.allclose(R, g.R, rtol=1e-14, atol=0) and R[0] > 0 and R[-1] < 1
    assert np.allclose(chi, g.chi, rtol=1e-15, atol=0)
    Tg = plan.basis()
    scale = np.abs(To).max(axis=-1, keepdims=True)
    scale[scale == 0] = 1.0
    assert np.max(np.abs(Tg - To) / scale) < TOL_BASIS


def test_cl_fp64_fp32_against_oracle(case):
    name, spec, g, To, plan = case
    L = spec.ells.size
    counts = [(spec.max_clust, spec.max_lens), (1, 0), (0, 2), (2, 1)]
    sels = [None, [0, L - 1], None, list(range(1, L, 2))]
    for i, ((ng, ns), sel) in enumerate(zip(counts, sels)):
        ng, ns = min(ng, spec.max_clust), min(ns, spec.max_lens)
        rq = subset_request(synth.config_request(name, g.chi, g.R, 60 + i), ng, ns, spec.max_clust)
        Co = _oracle(g, To, rq, sel)
        C64 = plan.cl(rq, bl.BLAST_FP64, ell_sel=sel)
        assert np.max(eij(C64, Co, ng, ns)) < TOL_FP64
        C32 = plan.cl(rq, bl.BLAST_FP32, ell_sel=sel)
        assert np.max(eij(C32, Co, ng, ns)) < TOL_FP32
    # a batch of uneven requests gives each request's own result
    rqs = [subset_request(synth.config_request(name, g.chi, g.R, 70 + i), ng, ns, spec.max_clust)
           for i, (ng, ns) in enumerate([(1, 1), (spec.max_clust, spec.max_lens), (0, 1)])]
    outs = plan.cl_batch(rqs, bl.BLAST_FP64)
    for rq, C in zip(rqs, outs):
        assert np.array_equal(C, plan.cl(rq, bl.BLAST_FP64))


def test_noalloc_and_refusals(case):
    import torch
    name, spec, g, To, plan = case
    rq = synth.config_request(name, g.chi, g.R, 5)
    fields = ["kern_chi", "kern_Rchi", "growth_chi", "growth_Rchi", "k_tab", "p_tab"]
    dev = {f: torch.from_numpy(np.ascontiguousarray(getattr(rq, f))).cuda() for f in fields}
    r = plan.request(rq, device_arrays=dev)
    ref = plan.cl(rq, bl.BLAST_FP64)
    out = torch.empty(ref.shape, dtype=torch.float64, device="cuda")
    assert bl.blast_cl_noalloc(plan.h, r, out.data_ptr(), torch.cuda.current_stream().cuda_stream) == bl.BLAST_OK
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), ref)
    Pq = np.ones((plan.Q, plan.N))
    with pytest.raises(bl.BlastError) as ei:
        plan.nonsep(rq, Pq)
    assert ei.value.status == bl.BLAST_EINVAL


@pytest.mark.parametrize("name", ["tc", "tcg"])
def test_tensor_core_symmetrised(name):
    spec = dataclasses.replace(synth.plan_spec(name), r_form=1)
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map, r_form=1)
    To = g.basis()
    plan = bl.Plan(spec)
    try:
        plan.precompute(bl.BASIS_ALL)
        L = spec.ells.size
        counts = [(spec.max_clust, spec.max_lens), (1, 0), (0, 2), (2, 1), (spec.max_clust, 1)]
        sels = [None, [0, L - 1], None, list(range(1, L, 2)), None]
        rqs = [subset_request(synth.config_request(name, g.chi, g.R, 90 + i), min(ng, spec.max_clust),
                              min(ns, spec.max_lens), spec.max_clust) for i, (ng, ns) in enumerate(counts)]
        outs = plan.cl_batch(rqs, bl.BLAST_BF16S, sels)
        for rq, sel, C in zip(rqs, sels, outs):
            Co = _oracle(g, To, rq, sel)
            assert np.max(eij(C, Co, rq.n_clust, rq.n_lens)) < TOL_FP32
            C64 = plan.cl(rq, bl.BLAST_FP64, ell_sel=sel)
            assert np.max(eij(C64, Co, rq.n_clust, rq.n_lens)) < TOL_FP64
            assert np.array_equal(plan.cl(rq, bl.BLAST_BF16S, ell_sel=sel), C)
    finally:
        plan.close()
