"""Limber, extended Limber and the non-linear correction (Secs. 2.2, 3.2)
through the C ABI against the oracle.

- blast_cl_limber with the request's linear P, plain and extended, against
  oracle.limber fed oracle.limber_plin (two spline solvers, FP64): e_ij <= 1e-12;
- blast_cl_limber with a caller's table at the Limber points against the
  oracle on the same table;
- blast_cl_nonlinear: the correction vanishes when P_delta is the linear P
  (C_tot equals blast_cl), and equals the oracle's C^Limber(P_lin) when
  P_delta = 2 P_lin, for the FP64 and the tensor-core beyond-Limber parts;
- blast_limber_k returns (l + 1/2) / chi.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2410_03632_gb300 import blast as bl
from paper_2410_03632_gb300 import synth
from tests.metrics import eij

pytestmark = pytest.mark.gpu


def _have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


if not _have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def case():
    spec = synth.plan_spec("tc")
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)
    plan = bl.Plan(spec)
    plan.precompute(bl.BASIS_ALL)
    rqs = [synth.config_request("tc", g.chi, g.R, i) for i in range(3)]
    yield spec, g, plan, rqs
    plan.close()


def _rel(C, ref):
    return float(np.max(np.abs(C - ref) / np.max(np.abs(ref), axis=1, keepdims=True)))


def test_limber_points(case):
    spec, g, plan, rqs = case
    k = bl.blast_limber_k(plan.h, spec.ells.size, spec.n_chi)
    assert np.array_equal(k, (spec.ells[:, None] + 0.5) / g.chi[None, :])


def test_limber_linear_plain_and_extended(case):
    spec, g, plan, rqs = case
    for rq in rqs:
        P = g.limber_plin(rq.growth_chi, rq.k_tab, rq.p_tab)
        for ext in (False, True):
            C = plan.limber(rq, extended=ext)
            Co = g.limber(rq.n_clust, rq.n_lens, rq.kern_chi, rq.growth_chi, P, extended=ext)
            assert np.max(eij(C, Co, rq.n_clust, rq.n_lens)) < 1e-12
            assert _rel(C, Co) < 1e-12


def test_limber_with_a_table_and_subsets(case):
    spec, g, plan, rqs = case
    rq = rqs[1]
    P = 1.3 * g.limber_plin(rq.growth_chi, rq.k_tab, rq.p_tab) * (1.0 + 0.1 * np.sin(g.chi[None, :] / 300.0))
    sel = [0, 4, spec.ells.size - 1]
    C = plan.limber(rq, p_nl=P, ell_sel=sel)
    Co = g.limber(rq.n_clust, rq.n_lens, rq.kern_chi, rq.growth_chi, P[sel], ell_subset=g.ells[sel])
    assert _rel(C, Co) < 1e-12
    with pytest.raises(bl.BlastError) as ei:  # extended needs the growth-separable linear P
        plan.limber(rq, p_nl=P, extended=True)
    assert ei.value.status == bl.BLAST_EINVAL


@pytest.mark.parametrize("prec", [bl.BLAST_FP64, bl.BLAST_BF16S])
def test_nonlinear_correction(case, prec):
    spec, g, plan, rqs = case
    for rq in rqs:
        Plin = g.limber_plin(rq.growth_chi, rq.k_tab, rq.p_tab)
        Clin = plan.cl(rq, prec)
        same = plan.nonlinear(rq, Plin, prec)
        scale = np.max(np.abs(g.limber(rq.n_clust, rq.n_lens, rq.kern_chi, rq.growth_chi, Plin)), axis=1,
                       keepdims=True)
        assert np.max(np.abs(same - Clin) / scale) < 1e-12
        tot = plan.nonlinear(rq, 2.0 * Plin, prec)
        Co = g.limber(rq.n_clust, rq.n_lens, rq.kern_chi, rq.growth_chi, Plin)
        assert np.max(np.abs((tot - Clin) - Co) / scale) < 1e-12
