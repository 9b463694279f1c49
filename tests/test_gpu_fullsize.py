"""Parity at the benchmark sizes, through the C ABI.

- The plain FP64 1+1-bin grid (16 ells to 200, n_chi = n_R = 64, order 32,
  65 537 k nodes) at full size, sampled at four ells: FP64 and tensor-core C_l
  of two cosmologies against the oracle.
- The 3x2pt 5+5-bin benchmark grid (64 ells to 1000, n_chi = n_R = 128, order
  64, 65 537 k nodes), in the batch configuration the benchmark times: the
  oracle computes the basis and C_l at l = 2 (a sampled output: every spectrum
  of one ell); the GPU basis, FP64 C_l and tensor-core C_l of a batch of
  cosmologies are compared with it.
- The 10+10-bin grid's shapes (20 tracers, 210 spectra, order 96, n_R = 192)
  on a few ells and chi nodes: FP64 and tensor-core C_l against the oracle for
  every spectrum and ell.
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


def _grid(spec):
    return orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                    spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)


def test_benchmark_grid_sampled_at_ell_2():
    spec = synth.plan_spec("c1")
    plan = bl.Plan(spec)
    try:
        plan.precompute(bl.BASIS_ALL)
        g = _grid(spec)
        To = g.basis(ell_subset=g.ells[:1])                     # [3][1][N][Q], l = 2
        Tg = plan.basis()[:, :1]
        scale = np.max(np.abs(To), axis=-1, keepdims=True)
        # the integrand oscillates as j_l(k chi) with k chi up to ~7e4, so the two
        # sides agree this well only because their nodes are the same IEEE values
        db = float(np.max(np.abs(Tg - To) / np.where(scale > 0, scale, 1.0)))
        print(f"\nbenchmark grid, l = 2: device basis vs oracle {db:.3e} of the row maximum")
        assert db < 1e-11
        chi, R, _ = plan.nodes()
        rqs = [synth.config_request("c1", chi, R, 1 + i) for i in range(8)]
        c64 = plan.cl_batch(rqs, bl.BLAST_FP64)
        ctc = plan.cl_batch(rqs, bl.BLAST_BF16S)
        for rq, a, b in zip(rqs, c64, ctc):
            Co = g.cl(To, g.fit(rq.k_tab, rq.p_tab), 5, 5, rq.kern_chi, rq.kern_Rchi, rq.growth_chi,
                      rq.growth_Rchi, ell_subset=g.ells[:1])
            assert np.max(eij(a[:, :1], Co, 5, 5)) < 1e-10
            assert np.max(eij(b[:, :1], Co, 5, 5)) < 1e-4
    finally:
        plan.close()


def test_ten_plus_ten_bin_shapes_fp64():
    spec = synth.plan_spec("c2s")
    plan = bl.Plan(spec)
    try:
        plan.precompute(bl.BASIS_ALL)
        g = _grid(spec)
        To = g.basis()
        chi, R, _ = plan.nodes()
        rqs = [synth.config_request("c2s", chi, R, i) for i in range(3)]
        outs = plan.cl_batch(rqs, bl.BLAST_FP64)
        otc = plan.cl_batch(rqs, bl.BLAST_BF16S)
        for rq, C, Ct in zip(rqs, outs, otc):
            assert C.shape == (210, spec.ells.size)
            Co = g.cl(To, g.fit(rq.k_tab, rq.p_tab), 10, 10, rq.kern_chi, rq.kern_Rchi, rq.growth_chi,
                      rq.growth_Rchi)
            assert np.max(eij(C, Co, 10, 10)) < 1e-10
            assert np.max(eij(Ct, Co, 10, 10)) < 1e-4
    finally:
        plan.close()


def test_one_plus_one_bin_grid_sampled_at_four_ells():
    spec = synth.plan_spec("c0")
    plan = bl.Plan(spec)
    try:
        plan.precompute(bl.BASIS_ALL)
        g = _grid(spec)
        sel = [0, 6, 11, 15]                                   # l = 2, 13, 59, 200
        To = g.basis(ell_subset=g.ells[sel])
        chi, R, _ = plan.nodes()
        rqs = [synth.config_request("c0", chi, R, i) for i in range(2)]
        c64 = plan.cl_batch(rqs, bl.BLAST_FP64, [sel, sel])
        ctc = plan.cl_batch(rqs, bl.BLAST_BF16S, [sel, sel])
        for rq, a, b in zip(rqs, c64, ctc):
            Co = g.cl(To, g.fit(rq.k_tab, rq.p_tab), 1, 1, rq.kern_chi, rq.kern_Rchi, rq.growth_chi,
                      rq.growth_Rchi, ell_subset=g.ells[sel])
            assert a.shape == Co.shape == (3, 4)
            assert np.max(eij(a, Co, 1, 1)) < 1e-10
            assert np.max(eij(b, Co, 1, 1)) < 1e-4
    finally:
        plan.close()



def test_high_ell_basis_and_cl():
    """Bessel recurrences and Miller normalisation at l up to 1999 (the 10+10-bin
    grid's range), on a grid small enough for the oracle."""
    spec = synth.PlanSpec(np.array([200, 600, 1000, 1999], np.int32), 8, 26.0, 4100.0, 32, 0.2, 1.8, 32,
                          1e-4, 1.0, 1, synth.kquad_points(1e-4, 1.0, 4100.0, 1.8), 1, 1)
    plan = bl.Plan(spec)
    try:
        plan.precompute(bl.BASIS_ALL)
        g = _grid(spec)
        To = g.basis()
        Tg = plan.basis()
        scale = np.max(np.abs(To), axis=-1, keepdims=True)
        assert np.max(np.abs(Tg - To) / np.where(scale > 0, scale, 1.0)) < 1e-11
        chi, R, _ = plan.nodes()
        rq = synth.make_request(chi, R, 1, 1)
        C = plan.cl(rq, bl.BLAST_FP64)
        Co = g.cl(To, g.fit(rq.k_tab, rq.p_tab), 1, 1, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi)
        # at l = 1999 eight chi nodes leave C ~ 1e-18 of cancelled sums (negative
        # autos): ill-conditioned, so the spectra are compared up to l = 1000
        assert np.max(eij(C[:, :3], Co[:, :3], 1, 1)) < 1e-10
    finally:
        plan.close()
