"""The random-gather probe (rddmc_gather_probe) that measures the denominator
of the walk's gather roofline: its table is one cycle through every row, so
each thread's chain of dependent loads visits rows all over the footprint."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1709_10187_gb300 import build as B  # noqa: E402
from paper_1709_10187_gb300 import rddmc as R  # noqa: E402

pytestmark = pytest.mark.gpu


def _cycle_length(nxt):
    seen = np.zeros(len(nxt), dtype=bool)
    r, n = 0, 0
    while not seen[r]:
        seen[r] = True
        r = int(nxt[r])
        n += 1
    return n, r


@pytest.mark.parametrize("rows,rb", [(64, 8), (4096, 8), (4096, 16), (1 << 17, 16)])
def test_probe_table_is_a_single_cycle(rows, rb):
    B.build()
    buf = torch.zeros(rows * rb, dtype=torch.uint8, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    n = R.gather_probe(buf.data_ptr(), rows * rb, rb, False, 64, 0, 256, 3, True, sink.data_ptr(), s)
    torch.cuda.synchronize()
    assert n % (64 * 256) == 0 and n >= 64 * 256 * 152
    words = buf.view(torch.int32).cpu().numpy().view(np.uint32).reshape(rows, rb // 4)
    nxt = words[:, 0].astype(np.int64)
    assert nxt.min() >= 0 and nxt.max() < rows
    length, back = _cycle_length(nxt)
    assert length == rows and back == 0


def test_probe_rates_are_ordered_by_footprint():
    # shared memory and L1-resident chains are served faster than HBM-bound ones
    B.build()
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    rates = {}
    for name, nbytes, smem, chain in (("l1", 32 << 10, False, 4096), ("smem", 32 << 10, True, 4096),
                                      ("hbm", 256 << 20, False, 256)):
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        R.gather_probe(buf.data_ptr(), nbytes, 8, smem, chain, 0, 256, 1, True, sink.data_ptr(), s)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        n = R.gather_probe(buf.data_ptr(), nbytes, 8, smem, chain, 0, 256, 2, False, sink.data_ptr(), s)
        a1.record()
        torch.cuda.synchronize()
        rates[name] = n / (a0.elapsed_time(a1) / 1e3)
    assert rates["l1"] > rates["hbm"] and rates["smem"] > rates["hbm"], rates
