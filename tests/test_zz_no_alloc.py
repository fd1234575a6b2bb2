"""kps_matvec_A_static_scratch: the allocation-free A*y for BF16/FP16 vectors.

It is compared with kps_matvec_A on the same inputs, on two calls in a row
with different inputs and batch sizes, so that the second call runs over the
first call's leftovers in the shared static array:
  - against kps_matvec_A on the same kernel (scalar staging), bit for bit;
  - against kps_matvec_A on its default kernel within 2 * TOL, since each
    output is within the parity bound TOL (2^-8 BF16, 2^-10 FP16, normwise:
    one rounding of the output) of the exact product;
  - the second call against the FP64 oracle on the same rounded inputs,
    within TOL.
The file is named to be collected last: it must pass both alone in a fresh
process and after every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.oracle import OracleGame
from paper_2112_03804_gb300 import kps, synth
from tests.gpu_util import from_library, library_order, normwise_error, to_library

pytestmark = pytest.mark.gpu

TOL = {kps.BF16: 2.0 ** -8, kps.F16: 2.0 ** -10}
TDT = {kps.BF16: torch.bfloat16, kps.F16: torch.float16}


@pytest.fixture(scope="module")
def river():
    spec = synth.river_spec(seed=2)
    g = kps.Game(spec)
    g.upload()
    torch.cuda.synchronize()
    return spec, g, library_order(spec["strength"])


def _vectors(g, order, batch, seed, dt):
    inf = g.info()
    v = synth.simplex_vectors(g.sequences(1)["nact"], inf["H"], batch, seed=seed)
    return torch.from_numpy(to_library(v, order, inf["hs"])).to("cuda", TDT[dt]).contiguous()


def _max_batch(g):
    inf = g.info()
    return kps.STATIC_SCRATCH_FLOATS // (inf["n1"] * inf["hs"])


def _host(t):
    return t.to(torch.float64).cpu().numpy()


@pytest.mark.parametrize("dt", [kps.BF16, kps.F16])
def test_two_calls_match_matvec_A(river, dt, monkeypatch):
    spec, g, order = river
    inf = g.info()
    # the largest batch that fits the static array, then a smaller one
    batches = [_max_batch(g), 17]
    ys = [_vectors(g, order, b, seed=101 + i, dt=dt) for i, b in enumerate(batches)]
    outs = [torch.full((b, inf["n1"], inf["hs"]), float("nan"), device="cuda", dtype=TDT[dt]) for b in batches]
    for y, out in zip(ys, outs):
        kps.matvec_A_static_scratch(g, y, out, y.shape[0], dtype=dt)
    refs = {}
    for kernel in ("default", "fast"):
        if kernel == "fast":
            monkeypatch.setenv("KPS_KERNEL", "fast")
        refs[kernel] = [torch.full_like(o, float("nan")) for o in outs]
        for y, ref in zip(ys, refs[kernel]):
            kps.matvec_A(g, y, ref, y.shape[0], dtype=dt)
    torch.cuda.synchronize()
    for i, out in enumerate(outs):
        o = _host(out)
        assert np.all(np.isfinite(o))
        assert np.all(o[..., inf["H"]:] == 0), "padding must be written as zero"
        assert np.array_equal(o, _host(refs["fast"][i]))
        assert normwise_error(o, _host(refs["default"][i])) <= 2 * TOL[dt]
    og = OracleGame(spec)
    got = from_library(_host(outs[1]), order, inf["H"])
    want = og.matvec_A(from_library(_host(ys[1]), order, inf["H"]))
    assert normwise_error(got, want) <= TOL[dt]


def test_no_device_memory_taken(river):
    """After the first call (which may load the kernel's module, and with it
    the static array), further calls leave the free device memory as it is."""
    spec, g, order = river
    inf = g.info()
    b = _max_batch(g)
    y = _vectors(g, order, b, seed=7, dt=kps.BF16)
    out = torch.empty((b, inf["n1"], inf["hs"]), device="cuda", dtype=torch.bfloat16)
    kps.matvec_A_static_scratch(g, y, out, b)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        kps.matvec_A_static_scratch(g, y, out, b)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_oversize_and_bad_arguments_rejected(river):
    spec, g, order = river
    inf = g.info()
    b = _max_batch(g) + 1
    y = torch.zeros((b, inf["n2"], inf["hs"]), device="cuda", dtype=torch.bfloat16)
    out = torch.zeros((b, inf["n1"], inf["hs"]), device="cuda", dtype=torch.bfloat16)
    with pytest.raises(kps.KpsError) as e:
        kps.matvec_A_static_scratch(g, y, out, b)
    assert e.value.status == kps.EINVAL and "exceeds the static scratch" in str(e.value)
    with pytest.raises(kps.KpsError) as e:
        kps.matvec_A_static_scratch(g, y.float(), out.float(), 1)
    assert e.value.status == kps.EINVAL
    fresh = kps.Game(spec)   # tables not uploaded: the call may not upload (that allocates)
    with pytest.raises(kps.KpsError) as e:
        kps.matvec_A_static_scratch(fresh, y, out, 1)
    assert e.value.status == kps.EINVAL


def test_refused_while_capturing(river):
    """The tile list is copied from host memory that lives only for the
    call, so a captured call would replay a dangling copy: the call refuses
    a capturing stream and queues nothing."""
    spec, g, order = river
    inf = g.info()
    y = _vectors(g, order, 2, seed=3, dt=kps.BF16)
    out = torch.zeros((2, inf["n1"], inf["hs"]), device="cuda", dtype=torch.bfloat16)
    kps.matvec_A_static_scratch(g, y, out, 2)     # device set-up outside the capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    status = None
    with torch.cuda.graph(graph, stream=side):
        try:
            kps.matvec_A_static_scratch(g, y, out, 2, stream=side)
        except kps.KpsError as e:
            status = e.status
    assert status == kps.EINVAL
    graph.replay()      # an empty graph
    torch.cuda.synchronize()
