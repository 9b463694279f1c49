"""Non-separable spectra through the C ABI against the oracle (FP64, e_ij <=
1e-10): a rank-two spectrum D1 D2 P_A + G1 G2 P_B sampled at the Chebyshev
k-nodes of every chi-R node, host and device samples, ell subsets; and a
separable input gives blast_cl's FP64 result."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as cheb

import oracle as orc
from paper_2410_03632_gb300 import blast as bl
from paper_2410_03632_gb300 import synth
from tests.metrics import eij

pytestmark = pytest.mark.gpu


def _torch_cuda():
    try:
        import torch
        return torch if torch.cuda.is_available() else None
    except Exception:
        return None


torch = _torch_cuda()
if torch is None:
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def case():
    spec = synth.plan_spec("small")
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)
    T = g.basis()
    plan = bl.Plan(spec)
    plan.precompute(bl.BLAST_BASIS_FP64)
    t, _ = orc.cheb_knodes(spec.n_cheb, spec.k_min, spec.k_max, spec.k_map)
    yield spec, g, T, plan, t
    plan.close()


def _rank_two(spec, g, rq, t):
    aA = g.fit(*synth.pk_table(-2.0, 0.05, 0.0, 0.8))
    aB = g.fit(*synth.pk_table(-1.6, 0.02, 1.0, 0.5))
    GB_chi, GB_R = 1.0 / (1.0 + g.chi / 3000.0), 1.0 / (1.0 + g.chi2 / 3000.0)
    return ((np.repeat(rq.growth_chi, spec.n_R) * rq.growth_Rchi)[:, None] * cheb.chebval(t, aA)[None, :]
            + (np.repeat(GB_chi, spec.n_R) * GB_R)[:, None] * cheb.chebval(t, aB)[None, :])


def test_nonsep_against_oracle(case):
    spec, g, T, plan, t = case
    for idx in range(2):
        rq = synth.config_request("small", g.chi, g.R, idx)
        Pq = _rank_two(spec, g, rq, t)
        ones = synth.Request(rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, np.ones_like(rq.growth_chi),
                             np.ones_like(rq.growth_Rchi), rq.k_tab, rq.p_tab)
        C = plan.nonsep(ones, Pq)
        Co = g.cl_nonsep(T, Pq, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi)
        assert np.max(eij(C, Co, rq.n_clust, rq.n_lens)) < 1e-10
        sel = [1, 5, spec.ells.size - 1]
        Cs = plan.nonsep(ones, Pq, ell_sel=sel)
        assert np.max(eij(Cs, Co[:, sel], rq.n_clust, rq.n_lens)) < 1e-10


def test_nonsep_device_samples_and_separable_input(case):
    spec, g, T, plan, t = case
    rq = synth.config_request("small", g.chi, g.R, 2)
    a = g.fit(rq.k_tab, rq.p_tab)
    Pq = (np.repeat(rq.growth_chi, spec.n_R) * rq.growth_Rchi)[:, None] * cheb.chebval(t, a)[None, :]
    fields = ["kern_chi", "kern_Rchi", "growth_chi", "growth_Rchi", "k_tab", "p_tab"]
    ones = synth.Request(rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, np.ones_like(rq.growth_chi),
                         np.ones_like(rq.growth_Rchi), rq.k_tab, rq.p_tab)
    dev = {f: torch.from_numpy(np.ascontiguousarray(getattr(ones, f))).cuda() for f in fields}
    dP = torch.from_numpy(np.ascontiguousarray(Pq)).cuda()
    out = torch.empty((bl.blast_npairs(rq.n_clust, rq.n_lens), spec.ells.size), dtype=torch.float64, device="cuda")
    r = plan.request(ones, device_arrays=dev)
    assert bl.blast_cl_nonsep(plan.h, r, dP.data_ptr(), out.data_ptr(), 1,
                              torch.cuda.current_stream().cuda_stream) == bl.BLAST_OK
    torch.cuda.synchronize()
    ref = plan.cl(rq, bl.BLAST_FP64)
    assert np.max(eij(out.cpu().numpy(), ref, rq.n_clust, rq.n_lens)) < 1e-10
