"""The top-k selection entry point that allocates nothing.

Callers that cannot allocate device memory at the moment they select (code
running while another component captures a CUDA graph, or a serving loop
whose device memory is all held by a pre-planned pool) call
rpq_topk_keys_noalloc; its intermediate buffers live in a fixed array inside
the library.  The array is shared by every call and keeps the previous call's
contents, so each check runs two calls in a row.  The reference is the
search's own CG selection (rpq_trace, the existing entry point) and, for a
large input, a plain sort.  This file is collected last on purpose."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _select(torch, rpq, keys: np.ndarray, k: int):
    d_keys = torch.from_numpy(keys.astype(np.uint32).view(np.int32)).cuda()
    d_out = torch.full((k,), -1, dtype=torch.int32, device="cuda")
    d_n = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rpq.topk_keys_noalloc(d_keys.data_ptr(), len(keys), k, d_out.data_ptr(), d_n.data_ptr(), stream)
    torch.cuda.synchronize()
    n = int(d_n.item())
    return d_out.cpu().numpy().view(np.uint32)[:n].copy()


def test_noalloc_matches_the_search_selection():
    import torch
    import paper_2001_06770_b300 as rpq
    import rpqgen
    ds = rpqgen.make_dataset("tiny")
    kg = rpq.KG.from_dataset(ds)
    try:
        for k in (10, 64):
            tr = kg.trace([124, 464], [], k, 6)
            cgs = tr["cgs"]                                   # (node << 8) | score
            keys = ((cgs & 0xff) << 26) | (cgs >> 8)          # (score << 26) | node
            assert len(keys) > k
            for _ in range(2):
                got = _select(torch, rpq, keys.astype(np.uint32), k)
                assert (got & ((1 << 26) - 1)).tolist() == tr["selected"].tolist()
                assert (got >> 26).tolist() == tr["results"]["s_c"].tolist()
    finally:
        kg.close()


def test_noalloc_large_input_then_small_input():
    import torch
    import paper_2001_06770_b300 as rpq
    rng = np.random.default_rng(7)
    big = rng.integers(0, 0xffffffff, size=3_000_000, dtype=np.uint64).astype(np.uint32)
    small = rng.integers(0, 0xffffffff, size=1000, dtype=np.uint64).astype(np.uint32)
    for keys in (big, small, big):
        got = _select(torch, rpq, keys, 64)
        assert got.tolist() == np.sort(keys)[:64].tolist()
    assert _select(torch, rpq, small[:5], 64).tolist() == np.sort(small[:5]).tolist()


def test_noalloc_rejects_out_of_range_arguments():
    import paper_2001_06770_b300 as rpq
    with pytest.raises(rpq.RPQError) as ei:
        rpq.topk_keys_noalloc(0x1000, (1 << 24) + 1, 10, 0x2000, 0x3000)
    assert ei.value.code == rpq.RPQ_ELIMIT
    with pytest.raises(rpq.RPQError) as ei:
        rpq.topk_keys_noalloc(0x1000, 100, 0, 0x2000, 0x3000)
    assert ei.value.code == rpq.RPQ_EINVAL
