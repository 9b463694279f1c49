"""The tcgen05 five-slice BF16 path against the FP64 oracle and the FP64 GPU path.

Bars: e_ij <= 1e-4 against the oracle and against the FP64 GPU result
(e_ij = |dC_ij| / sqrt(C_ii C_jj)); a cosmology's result is bitwise the same
alone and inside a batch; plans the kernel cannot serve are rejected.
"""
import numpy as np
import pytest

import oracle as orc
from paper_2410_03632_gb300 import blast as bl
from paper_2410_03632_gb300 import synth
from tests.metrics import eij

pytestmark = pytest.mark.gpu

TOL = 1e-4


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


@pytest.fixture(scope="module")
def tc_case():
    spec = synth.plan_spec("tc")
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)
    T = g.basis()
    plan = bl.Plan(spec)
    plan.precompute(bl.BASIS_ALL)
    yield spec, g, T, plan
    plan.close()


def oracle_cl(g, T, rq, sel=None):
    a = g.fit(rq.k_tab, rq.p_tab)
    Ts = T if sel is None else T[:, sel]
    return g.cl(Ts, a, rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi,
                ell_subset=None if sel is None else g.ells[sel])


def test_tc_matches_oracle_with_uneven_tracers_and_ells(tc_case):
    spec, g, T, plan = tc_case
    counts = [(3, 2), (1, 0), (0, 2), (2, 1), (3, 2), (1, 1)]
    L = spec.ells.size
    sels = [None, [0, 3], list(range(1, L, 2)), None, [L - 1], None]
    rqs = [subset_request(synth.config_request("tc", g.chi, g.R, i), ng, ns, spec.max_clust)
           for i, (ng, ns) in enumerate(counts)]
    outs = plan.cl_batch(rqs, bl.BLAST_BF16S, sels)
    for rq, s, C in zip(rqs, sels, outs):
        Co = oracle_cl(g, T, rq, s)
        assert C.shape == Co.shape
        assert np.max(eij(C, Co, rq.n_clust, rq.n_lens)) < TOL
        C64 = plan.cl(rq, bl.BLAST_FP64, ell_sel=s)
        assert np.max(eij(C, C64, rq.n_clust, rq.n_lens)) < TOL
        alone = plan.cl(rq, bl.BLAST_BF16S, ell_sel=s)
        assert np.array_equal(alone, C)  # a cosmology's row does not depend on its neighbours


def test_tc_two_ragged_cosmology_tiles(tc_case):
    spec, g, T, plan = tc_case
    base = [synth.config_request("tc", g.chi, g.R, i) for i in range(5)]
    rqs = [base[i % 5] for i in range(130)]  # 128 + 2: a second, mostly padded tile
    outs = plan.cl_batch(rqs, bl.BLAST_BF16S)
    for i in (0, 4, 127, 128, 129):
        C64 = plan.cl(rqs[i], bl.BLAST_FP64)
        assert np.max(eij(outs[i], C64, rqs[i].n_clust, rqs[i].n_lens)) < TOL
    assert np.array_equal(outs[0], outs[125]) and np.array_equal(outs[4], outs[129])


def test_tc_host_input_tiles_equal_device_input_batch(tc_case):
    """A batch of three cosmology tiles with host inputs (read in place over the
    host link) gives the bits of the same batch with device inputs."""
    import torch
    spec, g, T, plan = tc_case
    base = [synth.config_request("tc", g.chi, g.R, i) for i in range(9)]
    rqs = [base[i % 9] for i in range(300)]
    host = plan.cl_batch(rqs, bl.BLAST_BF16S)
    fields = ["kern_chi", "kern_Rchi", "growth_chi", "growth_Rchi", "k_tab", "p_tab"]
    dev = [{f: torch.from_numpy(np.ascontiguousarray(getattr(rq, f))).cuda() for f in fields} for rq in base]
    reqs = [plan.request(base[i % 9], device_arrays=dev[i % 9]) for i in range(300)]
    outs = [torch.empty(h.shape, dtype=torch.float64, device="cuda") for h in host]
    assert bl.blast_cl_batch(plan.h, reqs, bl.BLAST_BF16S, [o.data_ptr() for o in outs], 1,
                             torch.cuda.current_stream().cuda_stream) == bl.BLAST_OK
    torch.cuda.synchronize()
    for h, o in zip(host, outs):
        assert np.array_equal(h, o.cpu().numpy())


@pytest.mark.parametrize("n", [1, 31, 33, 64, 97])
def test_tc_partial_tiles_equal_full_batch(tc_case, n):
    """Batches that fill only some 32-lane quadrants of a tile (whose epilogue
    warps skip the padding) give every cosmology the bits it gets in a full
    tile of 128."""
    spec, g, T, plan = tc_case
    base = [synth.config_request("tc", g.chi, g.R, i) for i in range(7)]
    full = plan.cl_batch([base[i % 7] for i in range(128)], bl.BLAST_BF16S)
    part = plan.cl_batch([base[i % 7] for i in range(n)], bl.BLAST_BF16S)
    for i in range(n):
        assert np.array_equal(part[i], full[i])
    C64 = plan.cl(base[(n - 1) % 7], bl.BLAST_FP64)
    assert np.max(eij(part[n - 1], C64, spec.max_clust, spec.max_lens)) < TOL


@pytest.mark.parametrize("name", ["tcg", "tck"])
def test_tc_other_kernel_shapes(name):
    """The instances with tracer weights in two groups of five (7 + 6 tracers,
    weights of tracers 5.. in shared memory) and with the order past 64 (two K
    chunks per stage, four TMEM levels, the last holding slice levels 3 and 4)
    against the oracle, with uneven tracer counts and ell subsets."""
    spec = synth.plan_spec(name)
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)
    T = g.basis()
    plan = bl.Plan(spec)
    try:
        plan.precompute(bl.BASIS_ALL)
        mc, ml = spec.max_clust, spec.max_lens
        counts = [(mc, ml), (mc - 1, ml), (1, ml - 1), (mc, 0), (0, ml)]
        L = spec.ells.size
        sels = [None, [0, L - 1], None, list(range(1, L, 2)), None]
        rqs = [subset_request(synth.config_request(name, g.chi, g.R, i), ng, ns, mc)
               for i, (ng, ns) in enumerate(counts)]
        outs = plan.cl_batch(rqs, bl.BLAST_BF16S, sels)
        worst = 0.0
        for rq, s, C in zip(rqs, sels, outs):
            Co = oracle_cl(g, T, rq, s)
            assert C.shape == Co.shape
            worst = max(worst, float(np.max(eij(C, Co, rq.n_clust, rq.n_lens))))
            assert np.array_equal(plan.cl(rq, bl.BLAST_BF16S, ell_sel=s), C)
        print(f"\n{name}: worst e_ij against the oracle {worst:.3e}")
        assert worst < TOL
    finally:
        plan.close()


def test_tc_coefficient_envelope(tc_case):
    """The coefficient envelope only rescales both operands by powers of two:
    a flat envelope, the default one and a user shape all stay within 1e-4 of
    the oracle; a non-positive entry is refused."""
    spec, g, T, plan = tc_case
    rqs = [synth.config_request("tc", g.chi, g.R, i) for i in range(3)]
    ref = [oracle_cl(g, T, rq) for rq in rqs]
    try:
        for env in (np.ones(spec.n_cheb), 1.0 / (1.0 + np.arange(spec.n_cheb)) ** 2, None):
            assert bl.blast_set_coef_envelope(plan.h, env) == bl.BLAST_OK
            outs = plan.cl_batch(rqs, bl.BLAST_BF16S)
            for rq, C, Co in zip(rqs, outs, ref):
                assert np.max(eij(C, Co, rq.n_clust, rq.n_lens)) < TOL
        bad = np.ones(spec.n_cheb)
        bad[3] = 0.0
        assert bl.blast_set_coef_envelope(plan.h, bad) == bl.BLAST_EINVAL
    finally:
        bl.blast_set_coef_envelope(plan.h, None)


def test_tc_rejects_unsupported_plan():
    spec = synth.plan_spec("tiny")  # n_R = 10 is not a multiple of 32
    plan = bl.Plan(spec)
    plan.precompute(bl.BASIS_ALL)
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, 1025, spec.k_map)
    rq = synth.config_request("tiny", g.chi, g.R, 0)
    with pytest.raises(bl.BlastError) as ei:
        plan.cl_batch([rq, rq], bl.BLAST_BF16S)
    assert ei.value.status == bl.BLAST_EINVAL
    plan.close()


def test_tc_full_size_workload_against_fp64():
    """The 3x2pt 5+5-bin benchmark grid (64 ells to 1000, n_chi = n_R = 128,
    order 64): the five-slice path holds 1e-4 on every spectrum where the FP32
    path does not (high-l auto spectra of low-z lensing bins cancel strongly)."""
    spec = synth.plan_spec("c1")
    plan = bl.Plan(spec)
    plan.precompute(bl.BASIS_ALL)
    chi, R, _ = plan.nodes()
    rqs = [synth.config_request("c1", chi, R, 1 + i) for i in range(12)]
    outs = plan.cl_batch(rqs, bl.BLAST_BF16S)
    o64 = plan.cl_batch(rqs, bl.BLAST_FP64)
    worst = max(float(np.max(eij(a, b, 5, 5))) for a, b in zip(outs, o64))
    plan.close()
    assert worst < TOL, worst
