"""The launch-parameter autotuner of the tensor-core path: it picks a
contraction CTA count and a reduction shape on a representative batch, the
results stay within the tensor-core bar of the oracle, and the cache file
keyed by GPU, plan dimensions and cosmology tiles is written once and read
back by another plan without timing."""
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


def test_autotune_and_cache(tmp_path):
    spec = synth.plan_spec("tc")
    g = orc.Grid(spec.ells, spec.n_chi, spec.chi_min, spec.chi_max, spec.n_R, spec.R_min, spec.R_max,
                 spec.n_cheb, spec.k_min, spec.k_max, spec.n_kquad, spec.k_map)
    T = g.basis()
    cache = tmp_path / "tune.txt"
    plan = bl.Plan(spec)
    plan2 = bl.Plan(spec)
    try:
        plan.precompute(bl.BASIS_ALL)
        plan2.precompute(bl.BASIS_ALL)
        rqs = [synth.config_request("tc", g.chi, g.R, i) for i in range(6)]
        assert bl.blast_tuned_params(plan.h) == (0, 0, 0)
        assert bl.blast_autotune(plan.h, [plan.request(rq) for rq in rqs], cache) == bl.BLAST_OK
        params = bl.blast_tuned_params(plan.h)
        assert params[0] > 0 and params[1] in (2, 4, 8) and 1 <= params[2] <= 4
        outs = plan.cl_batch(rqs, bl.BLAST_BF16S)
        for rq, C in zip(rqs, outs):
            Co = g.cl(T, g.fit(rq.k_tab, rq.p_tab), rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi,
                      rq.growth_chi, rq.growth_Rchi)
            assert np.max(eij(C, Co, rq.n_clust, rq.n_lens)) < 1e-4
        lines = cache.read_text().splitlines()
        assert len(lines) == 1 and lines[0].endswith(" ".join(str(v) for v in params))
        assert bl.blast_autotune(plan2.h, [plan2.request(rq) for rq in rqs], cache) == bl.BLAST_OK
        assert bl.blast_tuned_params(plan2.h) == params
        assert len(cache.read_text().splitlines()) == 1
    finally:
        plan.close()
        plan2.close()
