"""Non-integer multipoles (App. A evaluates the basis at l = 211.63) through the
C ABI against the oracle's real-order Bessel functions.

Bars as for integer ells: basis within 1e-11 of its row maximum; FP64 C_l
within e_ij <= 1e-10, FP32 and the tensor-core path within 1e-4; Limber
within 1e-12; blast_limber_k returns (l + 1/2) / chi; integer values passed
as real multipoles give the integer plan's basis bit for bit.
"""
import dataclasses

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

REAL = {"tiny": np.array([2.5, 3.3, 7.75, 15.2, 40.63]),
        "tc": np.array([2.0, 3.7, 6.85, 12.67, 23.4, 43.3, 80.1, 148.2, 274.9])}


def _grid(spec):
    return orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                    spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)


@pytest.fixture(scope="module", params=["tiny", "tc"])
def case(request):
    name = request.param
    spec = dataclasses.replace(synth.plan_spec(name), ells=REAL[name])
    g = _grid(spec)
    To = g.basis()
    plan = bl.Plan(spec)
    plan.precompute(bl.BASIS_ALL)
    yield name, spec, g, To, plan
    plan.close()


def test_basis_at_real_ells(case):
    name, spec, g, To, plan = case
    Tg = plan.basis()
    scale = np.abs(To).max(axis=-1, keepdims=True)
    scale[scale == 0] = 1.0
    assert np.max(np.abs(Tg - To) / scale) < 1e-11


def test_cl_at_real_ells(case):
    name, spec, g, To, plan = case
    precs = [(bl.BLAST_FP64, 1e-10), (bl.BLAST_FP32, 1e-4)] + ([(bl.BLAST_BF16S, 1e-4)] if name == "tc" else [])
    for i in range(2):
        rq = synth.config_request(name, g.chi, g.R, 30 + i)
        a = g.fit(rq.k_tab, rq.p_tab)
        Co = g.cl(To, a, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi)
        for prec, tol in precs:
            C = plan.cl(rq, prec)
            assert np.max(eij(C, Co, rq.n_clust, rq.n_lens)) < tol, (prec,)


def test_limber_at_real_ells(case):
    name, spec, g, To, plan = case
    k = bl.blast_limber_k(plan.h, spec.ells.size, spec.n_chi)
    assert np.array_equal(k, (spec.ells[:, None] + 0.5) / g.chi[None, :])
    rq = synth.config_request(name, g.chi, g.R, 3)
    P = g.limber_plin(rq.growth_chi, rq.k_tab, rq.p_tab)
    C = plan.limber(rq)
    Co = g.limber(rq.n_clust, rq.n_lens, rq.kern_chi, rq.growth_chi, P)
    assert np.max(np.abs(C - Co) / np.max(np.abs(Co), axis=1, keepdims=True)) < 1e-12


def test_integer_values_as_real_multipoles_give_the_integer_plan():
    spec = synth.plan_spec("tiny")
    p_int = bl.Plan(spec)
    p_real = bl.Plan(dataclasses.replace(spec, ells=spec.ells.astype(np.float64)))
    try:
        p_int.precompute(bl.BASIS_ALL)
        p_real.precompute(bl.BASIS_ALL)
        assert np.array_equal(p_int.basis(), p_real.basis())
    finally:
        p_int.close()
        p_real.close()


def test_real_ells_in_the_symmetrised_form():
    """Both plan options at once: non-integer multipoles on the symmetrised
    chi-R form, FP64 against the oracle's symmetrised form at real ells."""
    spec = dataclasses.replace(synth.plan_spec("tiny"), ells=REAL["tiny"], r_form=1)
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map, r_form=1)
    To = g.basis()
    plan = bl.Plan(spec)
    try:
        plan.precompute(bl.BASIS_ALL)
        Tg = plan.basis()
        scale = np.abs(To).max(axis=-1, keepdims=True)
        scale[scale == 0] = 1.0
        assert np.max(np.abs(Tg - To) / scale) < 1e-11
        rq = synth.config_request("tiny", g.chi, g.R, 44)
        a = g.fit(rq.k_tab, rq.p_tab)
        Co = g.cl(To, a, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi)
        C = plan.cl(rq, bl.BLAST_FP64)
        assert np.max(eij(C, Co, rq.n_clust, rq.n_lens)) < 1e-10
    finally:
        plan.close()
