"""Failure detection without a GPU fault: host-side injection (AMR_FAULT) of a failed
device allocation and of a corrupted kD tree.  The corrupted root names itself as a child
but every index stays in range, so no access leaves its buffer: rays that loop at the root
stop at the descent's depth bound, set the device status word, and amr_render reports
AMR_ERR_DEVICE.  After either failure the same context builds and renders normally."""
import numpy as np
import pytest

import synth
from gpu_util import gpu_render, params_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amr():
    import paper_1212_3333_gb300 as m

    return m


@pytest.fixture(scope="module")
def c1():
    return synth.c1_workload()


def test_injected_device_allocation_failure(amr, c1, monkeypatch):
    from paper_1212_3333_gb300 import _lib

    w = c1
    ctx = amr.from_hierarchy(w["hier"])
    monkeypatch.setenv("AMR_FAULT", "oom")
    with pytest.raises(amr.AmrError) as e:
        ctx.amr_build_kdtree("ptr")
    assert e.value.status == _lib.AMR_ERR_OOM
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1)
    with pytest.raises(amr.AmrError) as e:  # nothing was uploaded
        gpu_render(ctx, w["camera"], w["tf"], p)
    assert e.value.status == _lib.AMR_ERR_STATE
    monkeypatch.delenv("AMR_FAULT")
    ctx.amr_build_kdtree("ptr")
    img, n = gpu_render(ctx, w["camera"], w["tf"], p)
    assert n > 0 and np.all(np.isfinite(img))


@pytest.mark.parametrize("schedule", [0, 3])
def test_injected_corrupt_tree_reports_a_device_error(amr, c1, monkeypatch, schedule):
    from paper_1212_3333_gb300 import _lib

    w = c1
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr", gradient=True)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, schedule=schedule)
    want, n_want = gpu_render(ctx, w["camera"], w["tf"], p)
    monkeypatch.setenv("AMR_FAULT", "corrupt_node")
    ctx.amr_build_kdtree("ptr", gradient=False)  # another storage variant: uploads again
    with pytest.raises(amr.AmrError) as e:
        gpu_render(ctx, w["camera"], w["tf"], p)
    assert e.value.status == _lib.AMR_ERR_DEVICE
    assert b"malformed" in ctx._lib.amr_last_error(ctx._h)
    monkeypatch.delenv("AMR_FAULT")
    ctx.amr_build_kdtree("ptr", gradient=True)
    img, n = gpu_render(ctx, w["camera"], w["tf"], p)
    assert n == n_want and np.array_equal(img, want)
