"""Failure detection on the GPU without a fault: the tensor-core kernels' bounded wait gives up on
an mbarrier that nothing completes, raises the CTA's abort flag so that the other wait returns at
once, frees TMEM and reports through the device status word; the context stays usable."""
import numpy as np
import pytest

import synth
from oracle import cg, topology
from tests.gpu_util import assert_close, require_gpu, to_dev, to_host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _gpu():
    require_gpu()


def test_bounded_wait_reports_and_context_stays_usable():
    from paper_2509_10226_gb300._lib import FemError
    from paper_2509_10226_gb300.fem import FemSpace

    p = 3
    xyz, cells = synth.kuhn_cube(4, jitter=0.2, seed=2)
    sp = FemSpace(xyz, cells, kind="cg", degree=p, device=0)
    assert sp.device_status() == 0
    limit = 0.05
    w0, w1 = sp.selftest_wait(limit)
    # the first wait ran to its limit; the second returned once the abort flag was raised
    assert limit <= max(w0, w1) < limit + 0.5
    assert min(w0, w1) < limit + 0.5
    assert sp.device_status() == 1
    assert sp.device_status() == 0  # read and cleared
    # the context (and its TMEM) is usable afterwards
    dofs, _ = topology.cg_numbering(cells, p)
    perm = sp.dof_permutation()
    u = synth.uniform_vector(sp.n_dofs, 1)
    y = to_host(sp.apply(to_dev(u[perm], "tf32"), prec="tf32"))
    assert_close(y, cg.apply(xyz, cells, u, p, dofs=dofs)[perm], "tf32", "apply after the self-test")
    assert sp.device_status() == 0
    with pytest.raises(FemError):
        sp.selftest_wait(0.0)
