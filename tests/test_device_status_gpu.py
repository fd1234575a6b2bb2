"""Failure detection on the device without a fault: a bounded wait that runs
out is reported by kps_device_status, and the context stays usable.

The TMA-staged kernel waits on an mbarrier for the copies of each box with a
limit of 2 s.  The test hook KPS_TEST_STALL_WAIT=1 makes one barrier per CTA
expect 16 bytes more than its copies bring (the copies themselves complete),
so that wait gives up: the warp stops scanning, the CTA drains and exits,
the kernel sets its flag, and kps_device_status returns KPS_ETIMEOUT once.
Then the same product, launched without the hook, is bit-identical to the
one before.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2112_03804_gb300 import kps, synth
from tests.gpu_util import library_order, to_library

pytestmark = pytest.mark.gpu


def test_wait_that_runs_out_is_reported(monkeypatch):
    spec = synth.river_spec(seed=2)
    g = kps.Game(spec)
    inf = g.info()
    B = 32                                   # one CTA per output sequence: a single wave
    v = synth.simplex_vectors(g.sequences(1)["nact"], inf["H"], B, seed=5)
    y = torch.from_numpy(to_library(v, library_order(spec["strength"]), inf["hs"])).to("cuda", torch.float32)
    out = [torch.zeros((B, inf["n1"], inf["hs"]), device="cuda") for _ in range(3)]
    monkeypatch.delenv("KPS_TEST_STALL_WAIT", raising=False)
    kps.matvec_A(g, y, out[0], B)
    kps.device_status()
    assert g.kernel(0) == "tma"
    monkeypatch.setenv("KPS_TEST_STALL_WAIT", "1")
    kps.matvec_A(g, y, out[1], B)
    with pytest.raises(kps.KpsError) as e:
        kps.device_status()
    assert e.value.status == kps.ETIMEOUT
    monkeypatch.delenv("KPS_TEST_STALL_WAIT")
    kps.device_status()                      # the flag was cleared
    kps.matvec_A(g, y, out[2], B)
    kps.device_status()
    assert torch.equal(out[2], out[0])
