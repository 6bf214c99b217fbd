"""Tile shapes of the EDT: every candidate shape gives the oracle's dt2 bit
for bit, autotuning keeps its choice per shape class (and in its cache
file), and bad arguments are refused."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2101_03240_gb300 import synth as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CANDIDATES = [(8, 16), (4, 16), (16, 16), (8, 8), (4, 8), (16, 8)]


@pytest.fixture(scope="module")
def ibip():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2101_03240_gb300 import ibip as m
    return m


def _cases():
    rng = np.random.default_rng(23)
    out = [S.blobs((37, 45, 29), 2.0, 0.6, rng), S.random_image((3, 70, 41), 0.9, rng),
           S.sphere_pack((33, 17, 130), 4, 0.45, rng), np.ones((9, 11, 13), np.uint8)]
    return out


@pytest.mark.parametrize("tile", CANDIDATES)
def test_every_tile_shape_matches_the_oracle(ibip, tile):
    ctx = ibip.Context(0)
    ctx.set_edt_tiles(*tile)
    for img in _cases():
        assert ctx.edt_tiles(img.shape) == tile
        got = ctx.edt(torch.from_numpy(img).cuda()).cpu().numpy()
        assert np.array_equal(got, O.edt(img)), (tile, img.shape)


def test_autotune_keeps_one_choice_per_shape_class(ibip, tmp_path):
    path = str(tmp_path / "tiles.txt")
    ctx = ibip.Context(0)
    ctx.set_autotune(True, path)
    img = _cases()[0]
    d = torch.from_numpy(img).cuda()
    got = ctx.edt(d).cpu().numpy()          # tunes, then computes
    assert np.array_equal(got, O.edt(img))
    lines = open(path).read().split("\n")
    lines = [ln for ln in lines if ln]
    assert len(lines) == 1 and lines[0].startswith("edt:6.6.5:sm")
    key, choice, us = lines[0].split()
    assert 0 <= int(choice) < len(CANDIDATES) and float(us) > 0
    assert ctx.edt_tiles(img.shape) == CANDIDATES[int(choice)]
    # the same class again: no new tuning line, the same result
    img2 = _cases()[0][:33, :40, :20].copy()
    assert np.array_equal(ctx.edt(torch.from_numpy(img2).cuda()).cpu().numpy(), O.edt(img2))
    assert len([ln for ln in open(path).read().split("\n") if ln]) == 1
    # a new context reading the file uses the stored choice
    ctx2 = ibip.Context(0)
    ctx2.set_autotune(True, path)
    assert ctx2.edt_tiles(img.shape) == CANDIDATES[int(choice)]
    # tuning off: the built-in shape
    ctx2.set_autotune(False)
    assert ctx2.edt_tiles(img.shape) == (8, 16)


def test_tile_arguments_are_checked(ibip):
    ctx = ibip.Context(0)
    with pytest.raises(ibip.IbipError):
        ctx.set_edt_tiles(12, 16)
    with pytest.raises(ibip.IbipError):
        ctx.set_edt_tiles(8, 0)
    ctx.set_edt_tiles(0, 0)
    assert ctx.edt_tiles((64, 64, 64)) == (8, 16)
    with pytest.raises(ibip.IbipError):
        ctx.set_autotune(True, "x" * 600)
    L = ibip._lib()
    assert L.ibip_set_autotune(ctx._h, 2, None) == ibip.ERR_ARG
