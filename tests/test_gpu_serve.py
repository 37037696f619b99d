"""The sort service on the GPU: every request's result, taken from the mixed
batches, equals the result of sorting that request alone, bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2206_01784_gb300 import onesweep as osw  # noqa: E402
from paper_2206_01784_gb300 import serve  # noqa: E402

pytestmark = pytest.mark.gpu


def test_each_result_same_alone_and_in_the_mix():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = serve.make_requests(160, seed=5, rate_per_s=20000.0, lo_log2=6, hi_log2=17)
    srv = serve.Server(budget_bytes=1 << 30, pool_words=1 << 22, keep_results=True)
    stats = srv.run(reqs, realtime=True)
    assert stats["requests"] == 160 and stats["batches"] >= 3
    assert stats["mean_batch_requests"] > 1.0  # requests really were coalesced
    dev = srv.device
    s = torch.cuda.current_stream().cuda_stream
    for r in reqs:
        kt = osw.KEY_TYPES[r.key_type]
        kb = serve.KEY_BYTES[r.key_type]
        raw = srv.request_input(r).to(dev)
        k = raw.view(torch.int64) if kb == 8 else raw
        v = torch.arange(r.n, dtype=torch.int32, device=dev)
        ko, vo = torch.empty_like(k), torch.empty_like(v)
        ws = osw.workspace(kt, r.n, 4, 0, 8 * kb, dev)
        assert osw.os_sort_pairs(kt, k.data_ptr(), ko.data_ptr(), v.data_ptr(), vo.data_ptr(), r.n, 0, 8 * kb,
                                 ws.data_ptr(), ws.numel(), s) == osw.OS_OK
        bk, bv = srv.result(r)
        torch.cuda.synchronize()
        assert torch.equal(bk, ko.view(torch.uint8)), r.rid
        assert torch.equal(bv, vo), r.rid
