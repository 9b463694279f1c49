"""The request server (continuous batching over resident plans) through the C ABI.

Bars: a request's C_l from the server equals the direct blast_cl result
(bitwise for FP64; for BF16S bitwise equal to the same request evaluated
alone), whatever else shares its batch; inputs are copied at submit (the
caller's arrays may go away); admission, tickets and bounded polls follow the
documented statuses; the reservation made at creation is checked against the
budget; plans served at once from several threads give the results each
request gets alone.
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


def subset_request(full, ng, ns, max_clust):
    kc = np.concatenate([full.kern_chi[:ng], full.kern_chi[max_clust:max_clust + ns]])
    kR = np.concatenate([full.kern_Rchi[:ng], full.kern_Rchi[max_clust:max_clust + ns]])
    return synth.Request(ng, ns, np.ascontiguousarray(kc), np.ascontiguousarray(kR), full.growth_chi,
                         full.growth_Rchi, full.k_tab, full.p_tab)


@pytest.fixture(scope="module")
def plans():
    out = []
    for name in ("tiny", "tc"):
        p = bl.Plan(synth.plan_spec(name))
        p.precompute(bl.BASIS_ALL)
        chi, R, _ = p.nodes()
        out.append((name, p, chi, R))
    yield out
    for _, p, _, _ in out:
        p.close()


@pytest.fixture(scope="module")
def more_tc():
    """Tensor-core plans of other shapes: 7 + 6 tracers (two tracer groups) and
    Chebyshev order 80 (two K chunks)."""
    out = []
    for name in ("tcg", "tck"):
        p = bl.Plan(synth.plan_spec(name))
        p.precompute(bl.BASIS_ALL)
        chi, R, _ = p.nodes()
        out.append((name, p, chi, R))
    yield out
    for _, p, _, _ in out:
        p.close()


def _cases(plans):
    """(plan index, request, precision, ell subset) for a mix of plans,
    precisions, tracer counts and ell subsets."""
    cases = []
    counts = [(3, 2), (1, 0), (0, 2), (2, 1), (3, 2), (1, 1)]
    for pi, (name, p, chi, R) in enumerate(plans):
        spec = p.spec
        L = p.L
        sels = [None, [0, L - 1], list(range(1, L, 2)), None, [L // 2], None]
        for i, (ng, ns) in enumerate(counts):
            ng, ns = min(ng, spec.max_clust), min(ns, spec.max_lens)
            if ng + ns == 0:
                continue
            rq = subset_request(synth.config_request(name, chi, R, 40 + i), ng, ns, spec.max_clust)
            cases.append((pi, rq, bl.BLAST_FP64, sels[i]))
            if name == "tc":
                cases.append((pi, rq, bl.BLAST_BF16S, sels[i]))
    return cases


def test_server_results_equal_direct_calls_in_a_mix(plans):
    cases = _cases(plans)
    refs = [plans[pi][1].cl(rq, prec, sel) for pi, rq, prec, sel in cases]  # before the server holds the plans
    srv = bl.Server([p for _, p, _, _ in plans], max_slots=5)
    try:
        tickets = []
        for pi, rq, prec, sel in cases:
            rc, t = srv.submit(pi, rq, prec, sel)
            assert rc == bl.BLAST_OK, bl.blast_status_str(rc)
            tickets.append(t)
        assert len(set(tickets)) == len(tickets)
        for (pi, rq, prec, sel), t, ref in zip(cases, tickets, refs):
            rc, C = srv.poll(t, ref.shape)
            assert rc == bl.BLAST_OK
            assert np.array_equal(C, ref)  # same bits alone and inside any batch
            assert srv.poll(t, ref.shape)[0] == bl.BLAST_EINVAL  # retired
    finally:
        srv.close()


def test_server_copies_device_inputs_at_submit(plans):
    import torch
    name, p, chi, R = plans[1]
    rq = synth.config_request(name, chi, R, 77)
    ref = p.cl(rq, bl.BLAST_FP64)
    srv = bl.Server([p], max_slots=4)
    try:
        fields = ["kern_chi", "kern_Rchi", "growth_chi", "growth_Rchi", "k_tab", "p_tab"]
        dev = {f: torch.from_numpy(np.ascontiguousarray(getattr(rq, f))).cuda() for f in fields}
        r = p.request(rq, device_arrays=dev)
        rc, t = bl.blast_submit(srv.h, 0, r, bl.BLAST_FP64)
        assert rc == bl.BLAST_OK
        for f in fields:  # overwrite the caller's arrays: the server holds its own copy
            dev[f].fill_(float("nan"))
        del r, dev
        torch.cuda.synchronize()
        rc, C = srv.poll(t, ref.shape)
        assert rc == bl.BLAST_OK and np.array_equal(C, ref)
    finally:
        srv.close()


def test_server_reservation_and_budget(plans):
    name, p, chi, R = plans[1]
    srv = bl.Server([p], max_slots=3)
    try:
        need = srv.reserved()
        # the ring (6 slots of the largest request) plus the plan's work space
        assert need > 6 * 8 * (p.spec.max_clust + p.spec.max_lens) * p.X
    finally:
        srv.close()
    with pytest.raises(bl.BlastError) as ei:
        bl.Server([p], hbm_budget=need - 1, max_slots=3)
    assert ei.value.status == bl.BLAST_ENOMEM
    srv = bl.Server([p], hbm_budget=need, max_slots=3)
    srv.close()
    with pytest.raises(bl.BlastError) as ei:  # a plan's work space serves one lane
        bl.Server([p, p], max_slots=3)
    assert ei.value.status == bl.BLAST_EINVAL


def test_server_admission_and_statuses(plans):
    name, p, chi, R = plans[1]
    spec = p.spec
    rq = synth.config_request(name, chi, R, 5)
    srv = bl.Server([p], max_slots=2)  # a ring of four device slots
    try:
        bad = synth.Request(spec.max_clust + 1, 0, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi,
                            rq.k_tab, rq.p_tab)
        assert srv.submit(0, bad, bl.BLAST_FP64)[0] == bl.BLAST_EINVAL
        # a P table that starts above the lowest Chebyshev node must be refused
        short = synth.Request(rq.n_clust, rq.n_lens, rq.kern_chi, rq.kern_Rchi, rq.growth_chi, rq.growth_Rchi,
                              np.ascontiguousarray(rq.k_tab * 10.0), rq.p_tab)
        assert short.k_tab[0] > p.nodes()[2].min()
        assert srv.submit(0, short, bl.BLAST_FP64)[0] == bl.BLAST_EINVAL
        assert srv.poll(123456789, (1, 1))[0] == bl.BLAST_EINVAL
        # a burst far faster than the GPU: the four slots must push back
        ok, busy = [], 0
        for _ in range(40):
            rc, t = srv.submit(0, rq, bl.BLAST_FP64)
            if rc == bl.BLAST_OK:
                ok.append(t)
            else:
                assert rc == bl.BLAST_EBUSY
                busy += 1
        assert busy > 0 and ok
        ref = None
        for t in ok:
            rc, C = srv.poll(t, (bl.blast_npairs(rq.n_clust, rq.n_lens), p.L), timeout_us=0)
            if rc == bl.BLAST_ENOTREADY:
                rc, C = srv.poll(t, (bl.blast_npairs(rq.n_clust, rq.n_lens), p.L), timeout_us=30_000_000)
            assert rc == bl.BLAST_OK
            ref = C if ref is None else ref
            assert np.array_equal(C, ref)
        # slots are free again once their batches ended
        rc, t = srv.submit(0, rq, bl.BLAST_FP64)
        assert rc == bl.BLAST_OK
        assert srv.poll(t, ref.shape, timeout_us=30_000_000)[0] == bl.BLAST_OK
        # BF16S on a plan the tensor-core kernel cannot serve
        tiny = plans[0][1]
        srv2 = bl.Server([tiny], max_slots=2)
        try:
            trq = synth.config_request("tiny", plans[0][2], plans[0][3], 1)
            assert srv2.submit(0, trq, bl.BLAST_BF16S)[0] == bl.BLAST_EINVAL
        finally:
            srv2.close()
    finally:
        srv.close()


def test_server_lanes_under_load_equal_alone(plans, more_tc):
    """Three tensor-core plans of different shapes (tracer groups, Chebyshev
    order) served at once from three submitting threads: every result equals
    the same request evaluated alone, bit for bit."""
    import threading
    lanes = [plans[1]] + more_tc
    work = []
    for li, (name, p, chi, R) in enumerate(lanes):
        rqs = [synth.config_request(name, chi, R, 300 + i) for i in range(6)]
        jobs = [(rqs[i % 6], bl.BLAST_BF16S if i % 3 else bl.BLAST_FP64) for i in range(48)]
        alone = {}
        for i, (rq, prec) in enumerate(jobs[:12]):
            alone[(i % 6, prec)] = p.cl(rq, prec)
        work.append((jobs, alone))
    srv = bl.Server([p for _, p, _, _ in lanes], max_slots=4)
    errors = []

    def client(li):
        jobs, alone = work[li]
        p = lanes[li][1]
        try:
            inflight = []
            for i, (rq, prec) in enumerate(jobs):
                while True:
                    rc, t = srv.submit(li, rq, prec)
                    if rc == bl.BLAST_OK:
                        break
                    assert rc == bl.BLAST_EBUSY
                    if inflight:  # drain the oldest to free a slot
                        j, tt = inflight.pop(0)
                        _check(li, j, tt)
                inflight.append((i, t))
            for j, tt in inflight:
                _check(li, j, tt)
        except Exception as e:  # surfaced in the main thread
            errors.append(e)

    def _check(li, j, t):
        jobs, alone = work[li]
        rq, prec = jobs[j]
        ref = alone[(j % 6, prec)]
        rc, C = srv.poll(t, ref.shape, timeout_us=60_000_000)
        assert rc == bl.BLAST_OK, bl.blast_status_str(rc)
        assert np.array_equal(C, ref)

    try:
        th = [threading.Thread(target=client, args=(li,)) for li in range(len(lanes))]
        for t in th:
            t.start()
        for t in th:
            t.join()
    finally:
        srv.close()
    assert not errors, errors[0]


def test_server_destroy_evaluates_waiting_requests(plans):
    name, p, chi, R = plans[1]
    rq = synth.config_request(name, chi, R, 9)
    srv = bl.Server([p], max_slots=2)
    for _ in range(4):
        assert srv.submit(0, rq, bl.BLAST_FP64)[0] == bl.BLAST_OK
    srv.close()  # returns after the waiting requests ran; nothing leaks or hangs
    assert p.cl(rq, bl.BLAST_FP64).shape[1] == p.L  # the plan is usable again
