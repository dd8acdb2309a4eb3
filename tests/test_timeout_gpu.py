"""A wait that runs out, without a GPU fault: the host-side bound of a polled step loop returns
MOTIF_ERR_TIMEOUT once its time is up, leaves nothing in flight, and the plan, the stream and the
context stay usable -- the same plan then finds the oracle's complete result.

The (15,4) workload on the per-candidate kernel takes many passes (four chunks of 2^28
candidates, one pass per sequence while candidates survive), so a 1 ms bound runs out after the
first group of polled steps.
"""
import json
import os

import numpy as np
import pytest

import paper_1403_1313_gb300 as m
from paper_1403_1313_gb300 import fmgen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "l15d4_n20_t600_seed2.json")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1403_1313_gb300 import build
    build.build()


def test_polled_batch_times_out_and_the_plan_recovers():
    with open(GOLDEN) as f:
        g = json.load(f)
    job = fmgen.single("l15d4")
    o = m.motif_opts_default()
    o.kernel = m.KERNEL_CAND
    o.timeout_ms = 1
    plan = m.motif_plan_create(job.n, job.t, job.l, job.d, o)
    m.motif_load_seqs(plan, job.seqs)
    with pytest.raises(m.MotifError) as e:
        m.motif_batch_search([plan], use_graph=False)
    assert e.value.status == m.ERR_TIMEOUT
    # the same plan, run to completion (the graph path bounds the loop by its step count only)
    got = m.motif_batch_search([plan], use_graph=True)[0]
    assert got.tolist() == g["codes"]
    assert np.array_equal(m.motif_search(plan), got)
    m.motif_plan_destroy(plan)
