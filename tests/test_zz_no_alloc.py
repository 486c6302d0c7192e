"""dtb_spike_compact_noalloc, the allocation-free compaction entry point.

It exists for callers that cannot allocate device memory while it runs (a
framework owning the whole device heap, a real-time loop that may not block
in cudaMalloc/cudaFree, a plugin handed only buffers).  Its scratch is a fixed
device array inside the library.  This test calls it through the C ABI twice
in a row, with different sizes, and checks each result against the
allocating entry point dtb_spike_compact on the same input.  Ids are
integers, so the tolerance is exact equality.  Kept in a file of its own that
pytest collects last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _device_bits(n, density, seed):
    import torch

    rng = np.random.default_rng(seed)
    flags = rng.random(n) < density
    pad = np.zeros(-(-n // 1024) * 1024, bool)
    pad[:n] = flags
    bits = np.packbits(pad, bitorder="little").view(np.uint32)  # bit b of word w = neuron 32w + b
    return torch.from_numpy(bits.view(np.int32)).cuda(), np.flatnonzero(flags)


def test_noalloc_matches_allocating_compaction_on_two_calls():
    import torch

    from paper_2308_01241_gb300 import dtb

    stream = torch.cuda.current_stream().cuda_stream
    for n, density, seed in [(3_000_001, 0.01, 1), (200_003, 0.3, 2)]:  # the second call is smaller
        bits, expect = _device_bits(n, density, seed)
        ids_ref = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        cnt_ref = torch.zeros(1, dtype=torch.int32, device="cuda")
        dtb.dtb_spike_compact(bits, n, ids_ref, cnt_ref, stream)
        ids = torch.full((n,), -2, dtype=torch.int32, device="cuda")
        cnt = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        dtb.dtb_spike_compact_noalloc(bits, n, ids, cnt, stream)
        torch.cuda.synchronize()
        c = int(cnt.item())
        assert c == int(cnt_ref.item()) == expect.size
        np.testing.assert_array_equal(ids[:c].cpu().numpy(), ids_ref[:c].cpu().numpy())
        np.testing.assert_array_equal(ids[:c].cpu().numpy(), expect)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch

    from paper_2308_01241_gb300 import dtb

    bits = torch.zeros(32, dtype=torch.int32, device="cuda")
    ids = torch.zeros(32, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(dtb.DtbError) as e:
        dtb.dtb_spike_compact_noalloc(bits, dtb.NOALLOC_MAX_NEURONS + 1, ids, cnt)
    assert e.value.code == dtb.DTB_EINVAL
    assert "fixed scratch" in str(e.value)
