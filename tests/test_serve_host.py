"""CPU checks of the serving scheduler's host logic (argument checks, admission against the
memory budget, tickets, poll timeouts).  Without a GPU every admitted request fails when its
engine is created, and that failure must come back through ks_serve_poll, not hang."""
import os

import pytest

from paper_2106_03872_gb300 import inputs


@pytest.fixture(scope="module")
def ks():
    from paper_2106_03872_gb300 import ks as mod
    if not os.path.exists(mod.LIB_PATH):
        from paper_2106_03872_gb300 import build
        build.build()
    mod.load()
    return mod


def test_submit_argument_checks(ks):
    srv = ks.Server(1 << 30)
    cell = inputs.small_cell(10.0, 24, 2, 4, 1)
    for kind, count, dt in [(2, 1, 0.05), (0, -1, 0.05), (1, 3, 0.0), (1, 3, 50.0)]:
        with pytest.raises(ks.KsError) as e:
            srv.submit(cell, kind, count, dt)
        assert e.value.status == ks.KS_ERR_ARG
    with pytest.raises(ks.KsError) as e:
        srv.submit(dict(cell, N=25), 0, 1)
    assert e.value.status == ks.KS_ERR_ARG
    srv.close()


def test_request_above_budget_is_rejected(ks):
    srv = ks.Server(256 << 20)
    with pytest.raises(ks.KsError) as e:
        srv.submit(inputs.cell("td128"), 1, 2)
    assert e.value.status == ks.KS_ERR_NOMEM
    srv.close()


def test_unknown_ticket(ks):
    srv = ks.Server(1 << 30)
    st, _, _, _ = srv.poll(12345, 0)
    assert st == ks.KS_ERR_ARG
    srv.close()


def test_requests_complete_or_fail_without_hanging(ks):
    """Every ticket resolves: KS_OK with a GPU, an error status without one."""
    import torch
    srv = ks.Server(1 << 30)
    cell = inputs.small_cell(10.0, 24, 2, 4, 1)
    tickets = [srv.submit(cell, k % 2, 2) for k in range(4)]
    for t in tickets:
        st = ks.KS_PENDING
        for _ in range(600):
            st, _, _, _ = srv.poll(t, 100)
            if st not in (ks.KS_PENDING, ks.KS_ERR_TIMEOUT):
                break
        if torch.cuda.is_available():
            assert st == ks.KS_OK
        else:
            assert st in (ks.KS_ERR_CUDA, ks.KS_ERR_NOMEM)
            assert b"request failed" in ks.load().ks_last_error()
    # the counters: every request was started once, and the parts of the start time add up to
    # at most the start time itself
    stats = srv.stats()
    assert len(stats) == 14 and stats["starts"] == 4
    parts = stats["start_create_s"] + stats["start_init_s"] + stats["start_orthonormalize_s"]
    assert 0.0 <= parts <= stats["start_s"] + 1e-9
    assert stats["pool_slabs_allocated"] >= 0 and stats["pool_alloc_s"] >= 0.0
    srv.close()
