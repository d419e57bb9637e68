"""Failure detection without a GPU fault: every wait inside an epoch kernel is bounded in time
(hp.wait_limit_us), and when one runs out the kernel records where, skips the tile's
updates, releases its tensor memory and returns; the epoch reports S3_ERR_CUDA, the context
is marked failed, and the device stays usable for a new context.  A wait limit of a few
microseconds makes the waits run out (nothing is broken: the hand-offs simply take longer
than that).  The device-memory cap (hp.device_bytes_cap) turns an allocation beyond it into
S3_ERR_OOM."""
import numpy as np
import pytest

from paper_1708_08640_gb300 import _lib as L
from paper_1708_08640_gb300 import synth

pytestmark = pytest.mark.gpu


def _usable_after(p, prec, mode):
    """A fresh context on the same device runs the same epoch and stays finite."""
    from paper_1708_08640_gb300.model import S3CMTF
    m = S3CMTF.from_problem(p, order=synth.union_order(p, 2))
    m.set_params(*synth.init_params(p, 1))
    r0 = m.rmse(p.test_idx, p.test_val)
    m.epoch(mode, prec)
    r1 = m.rmse(p.test_idx, p.test_val)
    m.close()
    assert np.isfinite(r1) and r1 < r0


@pytest.mark.parametrize("J", [16, 32])
def test_tensor_core_wait_runs_out_and_is_reported(cuda_lib, J):
    """The BF16 kernel's MMA warp waits for the entry warps' operands for at most 2 us: it
    gives up at its first hand-off, the entry warps' waits run out in turn, and the epoch
    fails cleanly."""
    from paper_1708_08640_gb300.model import S3CMTF
    p = synth.with_rank(synth.make_problem("cfg1_tiny"), (J, J, J))
    m = S3CMTF.from_problem(p, order=synth.union_order(p, 2), wait_limit_us=2)
    m.set_params(*synth.init_params(p, 1))
    with pytest.raises(L.S3Error) as ei:
        m.epoch("hogwild", "bf16")
    assert ei.value.status == L.S3_ERR_CUDA
    assert "bounded wait ran out" in str(ei.value), str(ei.value)
    # the context is failed from now on
    with pytest.raises(L.S3Error) as ei2:
        m.loss()
    assert ei2.value.status == L.S3_ERR_STATE
    m.close()
    _usable_after(p, "bf16", "hogwild")


def test_grid_barrier_wait_runs_out_and_is_reported(cuda_lib):
    """The minibatch epoch's grid-wide barrier waits at most 1 us: CTAs that arrive early
    give up, every CTA leaves at its next barrier, and the epoch fails cleanly."""
    from paper_1708_08640_gb300.model import S3CMTF
    p = synth.make_problem("cfg1_small")
    m = S3CMTF.from_problem(p, order=synth.union_order(p, 2), wait_limit_us=1)
    m.set_params(*synth.init_params(p, 1))
    with pytest.raises(L.S3Error) as ei:
        m.epoch("minibatch")
    assert ei.value.status == L.S3_ERR_CUDA
    assert "grid barrier" in str(ei.value), str(ei.value)
    m.close()
    _usable_after(synth.make_problem("cfg1_tiny"), "fp32", "minibatch")


def test_device_memory_cap(cuda_lib):
    """A cap below what the layout needs fails s3_init with S3_ERR_OOM; a cap above it
    changes nothing."""
    from paper_1708_08640_gb300.model import S3CMTF
    p = synth.make_problem("cfg1_tiny")
    with pytest.raises(L.S3Error) as ei:
        S3CMTF.from_problem(p, device_bytes_cap=1 << 20)
    assert ei.value.status == L.S3_ERR_OOM
    a = S3CMTF.from_problem(p, order=synth.union_order(p, 2), device_bytes_cap=1 << 34)
    b = S3CMTF.from_problem(p, order=synth.union_order(p, 2))
    for m in (a, b):
        m.set_params(*synth.init_params(p, 1))
        m.epoch("minibatch")
    Ga, Ua, _ = a.get_params()
    Gb, Ub, _ = b.get_params()
    assert (Ga == Gb).all() and all((x == y).all() for x, y in zip(Ua, Ub))
    a.close()
    b.close()
