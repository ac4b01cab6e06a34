"""Allocation-free compaction entry point, checked against the render path's filter.

fgs_compact_selection_noalloc() serves callers that cannot allocate device memory
(a host application that owns all allocations, code running under stream capture,
a real-time loop).  It must return exactly the selection fgs_filter() returns for
the same selection bits, on two calls in a row (the second reuses the shared
static scratch left by the first).  This file sorts last so that a run stopping
at the first failure has already run every other test."""
import numpy as np
import pytest

from paper_2603_23891_gb300 import synth

pytestmark = pytest.mark.gpu


def _bits_of(ids, n_words):
    bits = np.zeros(n_words, np.uint32)
    np.bitwise_or.at(bits, ids // 32, (np.uint32(1) << (ids % 32).astype(np.uint32)))
    return bits


def test_noalloc_compaction_matches_filter():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_23891_gb300 import build, filtergs
    build.build()
    tree = synth.random_small_tree(5, n_leaves=20000, branching=(2, 8), sh_degree=0,
                                   extent=30.0, log_scale_mean=-0.8)
    r = filtergs.Renderer(device=0, tau_R=3.0)
    try:
        r.load_tree(tree)
        n_words = (tree.n + 31) // 32 + 5          # a ragged tail of empty words
        cams = [synth.look_at_camera([0, -60, 30], [0, 0, 0], 320, 240, 60.0),
                synth.look_at_camera([40, 40, 20], [0, 0, 0], 320, 240, 75.0)]
        for cam in cams:                             # two calls in a row
            r.set_camera(cam)
            ref = r.filter()                         # existing entry point
            assert ref.size > 100
            bits = torch.from_numpy(_bits_of(ref.astype(np.int64), n_words)).cuda()
            ids = torch.full((n_words * 32,), 0xFFFFFFFF, dtype=torch.int64).to(torch.int32).cuda()
            count = torch.zeros(1, dtype=torch.int32, device="cuda")
            stream = torch.cuda.current_stream().cuda_stream
            code = filtergs.fgs_compact_selection_noalloc(bits, n_words, ids, count, stream)
            assert code == filtergs.FGS_OK
            torch.cuda.synchronize()
            m = int(count.cpu().numpy().view(np.uint32)[0])
            assert m == ref.size
            got = ids[:m].cpu().numpy().view(np.uint32)
            assert np.array_equal(got, ref)
        # sizes beyond the stated maximum are rejected before any launch
        assert filtergs.fgs_compact_selection_noalloc(bits, (1 << 26) + 1, ids, count,
                                                      stream) == filtergs.FGS_ERR_ARG
    finally:
        r.close()


def test_noalloc_many_tiles_back_to_back():
    """Cross-tile look-back through the static scratch: 70, 23, 5 and 1 tiles (each
    with a ragged tail), dense, sparse and empty words, checked bit for bit against
    the set-bit positions computed on the host, every call."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_23891_gb300 import build, filtergs
    build.build()
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream().cuda_stream
    words_per_tile = 1024
    cases = [(70 * words_per_tile + 333, 0.5), (23 * words_per_tile + 17, 0.02),
             (5 * words_per_tile + 1, 0.9), (words_per_tile - 7, 0.3), (70 * words_per_tile, 0.0),
             (12 * words_per_tile + 500, 0.001)]
    for n_words, density in cases:
        bits01 = rng.random(n_words * 32) < density
        if density > 0:
            bits01[: 32 * 40] = True                 # a run of full words
            bits01[32 * 100: 32 * 300] = False       # a run of empty words
        words = np.packbits(bits01.reshape(-1, 32)[:, ::-1], axis=1).view(">u4").ravel().astype(np.uint32)
        expect = np.flatnonzero(bits01).astype(np.uint32)
        bits = torch.from_numpy(words.view(np.int32).copy()).cuda()
        ids = torch.full((n_words * 32,), -1, dtype=torch.int32, device="cuda")
        count = torch.zeros(1, dtype=torch.int32, device="cuda")
        code = filtergs.fgs_compact_selection_noalloc(bits, n_words, ids, count, stream)
        assert code == filtergs.FGS_OK
        torch.cuda.synchronize()
        m = int(count.cpu().numpy().view(np.uint32)[0])
        assert m == expect.size, (n_words, density, m, expect.size)
        got = ids[:m].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, expect), (n_words, density)
