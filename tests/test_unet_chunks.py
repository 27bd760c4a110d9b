"""Chunking of the combined comparison (host logic, no GPU): the chunks cover
every pair once, in order, ramping up from batch / 8 and batch / 2 pairs to
`batch`, so that only the first, small chunk's warm-start prediction is not
overlapped with solves."""

import pytest

from paper_2401_17493_b300.unet import combined_chunks


@pytest.mark.parametrize("npairs,batch,sizes", [
    (200, 64, [8, 32, 64, 64, 32]),
    (64, 64, [8, 32, 24]),
    (3, 64, [3]),
    (10, 4, [1, 2, 4, 3]),
    (5, 1, [1, 1, 1, 1, 1]),
])
def test_chunks_ramp_up_and_cover_every_pair_once(npairs, batch, sizes):
    chunks = combined_chunks(npairs, batch)
    assert [len(c) for c in chunks] == sizes
    assert [i for c in chunks for i in c] == list(range(npairs))
    assert max(len(c) for c in chunks) <= batch
