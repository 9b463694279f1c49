"""Parity of the CUDA path against the FP64 oracle, through the C ABI.

Bars: basis T~ elementwise within 1e-11 of the row maximum; FP64 C_l within
e_ij <= 1e-10 and FP32 C_l within e_ij <= 1e-4 of the oracle, with
e_ij = |dC_ij| / sqrt(C_ii C_jj) (auto-spectrum normalisation).
"""
import numpy as np
import pytest

import oracle as orc
from paper_2410_03632_gb300 import blast as bl
from paper_2410_03632_gb300 import synth
from tests.metrics import eij

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_MIXED = 1e-4
TOL_BASIS = 1e-11


def _have_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


if not _have_gpu():
    pytest.skip("needs a CUDA device", allow_module_level=True)


def oracle_grid(spec):
    return orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min,
                    spec.R_max, spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)


class Case:
    def __init__(self, name, basis_on_gpu=True):
        self.spec = synth.plan_spec(name)
        self.plan = bl.Plan(self.spec)
        self.g = oracle_grid(self.spec)
        self.To = self.g.basis()
        self.plan.precompute(bl.BASIS_ALL)
        self.name = name

    def request(self, idx=0):
        return synth.config_request(self.name, self.g.chi, self.g.R, idx)

    def oracle_cl(self, rq, T=None, ell_sel=None):
        a = self.g.fit(rq.k_tab, rq.p_tab)
        T = self.To if T is None else T
        if ell_sel is not None:
            T = T[:, ell_sel]
        return self.g.cl(T, a, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi,
                         rq.growth_Rchi, ell_subset=None if ell_sel is None else self.g.ells[ell_sel])


@pytest.fixture(scope="module", params=["tiny", "small"])
def case(request):
    c = Case(request.param)
    yield c
    c.plan.close()


def test_nodes_match_oracle(case):
    chi, R, kc = case.plan.nodes()
    assert np.allclose(chi, case.g.chi, rtol=1e-15, atol=0)
    assert np.allclose(R, case.g.R, rtol=1e-14, atol=0)
    _, ko = orc.cheb_knodes(case.spec.n_cheb, case.spec.k_min, case.spec.k_max, case.spec.k_map)
    assert np.allclose(kc, ko, rtol=1e-14, atol=0)


def test_basis_parity(case):
    Tg = case.plan.basis()
    To = case.To
    scale = np.abs(To).max(axis=-1, keepdims=True)
    scale[scale == 0] = 1.0
    err = np.abs(Tg - To) / scale
    assert np.max(err) < TOL_BASIS, np.max(err)


@pytest.mark.parametrize("prec,tol", [(bl.BLAST_FP64, TOL_FP64), (bl.BLAST_FP32, TOL_MIXED)])
def test_cl_end_to_end(case, prec, tol):
    rq = case.request(0)
    Cg = case.plan.cl(rq, prec)
    Co = case.oracle_cl(rq)
    e = eij(Cg, Co, rq.n_clust, rq.n_lens)
    assert np.max(e) < tol, np.max(e)


def test_cl_fed_oracle_basis(case):
    """Contraction + quadrature alone: the library given the oracle's T~."""
    spec = case.spec
    p = bl.Plan(spec)
    p.set_basis(case.To)
    rq = case.request(1)
    Cg = p.cl(rq, bl.BLAST_FP64)
    Co = case.oracle_cl(rq)
    p.close()
    assert np.max(eij(Cg, Co, rq.n_clust, rq.n_lens)) < TOL_FP64


def test_cl_ell_subset_and_tracer_counts(case):
    spec = case.spec
    L = spec.ells.size
    sel = [0, L - 1] if L > 1 else [0]
    for (ng, ns) in [(spec.max_clust, 0), (0, spec.max_lens), (1, 1)]:
        if ng + ns == 0:
            continue
        full = case.request(2)
        rq = synth.Request(ng, ns,
                           np.ascontiguousarray(np.concatenate([full.kern_chi[:ng], full.kern_chi[spec.max_clust:spec.max_clust + ns]])),
                           np.ascontiguousarray(np.concatenate([full.kern_Rchi[:ng], full.kern_Rchi[spec.max_clust:spec.max_clust + ns]])),
                           full.growth_chi, full.growth_Rchi, full.k_tab, full.p_tab)
        Cg = case.plan.cl(rq, bl.BLAST_FP64, ell_sel=sel)
        Co = case.oracle_cl(rq, ell_sel=sel)
        assert Cg.shape == (bl.blast_npairs(ng, ns), len(sel))
        assert np.max(eij(Cg, Co, ng, ns)) < TOL_FP64


@pytest.mark.parametrize("prec,tol", [(bl.BLAST_FP64, TOL_FP64), (bl.BLAST_FP32, TOL_MIXED)])
def test_batch_matches_single(case, prec, tol):
    rqs = [case.request(i) for i in range(3)]
    L = case.spec.ells.size
    sels = [None, [0], list(range(0, L, 2))]
    outs = case.plan.cl_batch(rqs, prec, sels)
    for rq, s, C in zip(rqs, sels, outs):
        Cs = case.plan.cl(rq, prec, ell_sel=s)
        if prec == bl.BLAST_FP64:
            assert np.array_equal(C, Cs)  # deterministic: alone == in a batch
        Co = case.oracle_cl(rq, ell_sel=s)
        assert np.max(eij(C, Co, rq.n_clust, rq.n_lens)) < tol


def test_invalid_requests_rejected(case):
    rq = case.request(0)
    keep = rq.k_tab > 3 * case.spec.k_min  # table no longer brackets the lowest Chebyshev node
    bad = synth.Request(rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi,
                        np.ascontiguousarray(rq.k_tab[keep]), np.ascontiguousarray(rq.p_tab[keep]))
    with pytest.raises(bl.BlastError) as ei:
        case.plan.cl(bad)
    assert ei.value.status == bl.BLAST_EINVAL
    too_many = synth.Request(case.spec.max_clust + 1, 0, rq.kern_chi, rq.kern_Rchi, rq.growth_chi,
                             rq.growth_Rchi, rq.k_tab, rq.p_tab)
    with pytest.raises(bl.BlastError):
        case.plan.cl(too_many)
    neg = synth.Request(rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi,
                        rq.k_tab, -rq.p_tab)
    with pytest.raises(bl.BlastError):
        case.plan.cl(neg)


def test_basis_save_load_roundtrip(case, tmp_path):
    path = str(tmp_path / "basis.bin")
    bl.blast_basis_save(case.plan.h, path)
    p2 = bl.Plan(case.spec)
    bl.blast_basis_load(p2.h, path, bl.BASIS_ALL)
    assert np.array_equal(p2.basis(), case.plan.basis())
    rq = case.request(0)
    assert np.array_equal(p2.cl(rq), case.plan.cl(rq))
    p2.close()
    other = synth.plan_spec("tiny" if case.name == "small" else "small")
    p3 = bl.Plan(other)
    with pytest.raises(bl.BlastError):
        bl.blast_basis_load(p3.h, path, bl.BASIS_ALL)
    p3.close()
