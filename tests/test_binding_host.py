"""Host-side logic of the Python binding that needs no GPU: the tile autotuner's JSON cache (a stored
result for the same device, d and nmax is reused; anything else is ignored) and the argument checks of
steady_state_batched's tile table."""
import json

import pytest
import torch

import paper_2608_30860_b300 as B


def _fake_device(monkeypatch, name="Fake B300"):
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda dev=None: name)


def _entry(name="Fake B300", d=2, nmax=160, tiles=None):
    return {"device": name, "d": d, "nmax": nmax, "shapes": list(B.TILE_NAMES),
            "tiles": tiles if tiles is not None else [2] * B.LB_TILE_BUCKETS, "us": [], "buckets": []}


def test_matching_cache_entry_is_reused_without_the_library(monkeypatch, tmp_path):
    _fake_device(monkeypatch)
    monkeypatch.setattr(B.lindblad, "load_library", lambda *a, **k: pytest.fail("the cache hit must not tune"))
    path = tmp_path / "tiles.json"
    path.write_text(json.dumps(_entry()))
    got = B.batched_tune(2, nmax=160, cache=str(path))
    assert got["cached"] and got["tiles"] == [2] * B.LB_TILE_BUCKETS


@pytest.mark.parametrize("entry", [
    _entry(name="Other GPU"), _entry(d=3), _entry(nmax=96), _entry(tiles=[0] * 3), _entry(tiles=[9] * 16),
    "not json at all {",
])
def test_mismatched_or_malformed_cache_is_not_used(monkeypatch, tmp_path, entry):
    _fake_device(monkeypatch)

    class Tuned(Exception):
        pass

    def no_library(*a, **k):
        raise Tuned()
    monkeypatch.setattr(B.lindblad, "load_library", no_library)
    path = tmp_path / "tiles.json"
    path.write_text(entry if isinstance(entry, str) else json.dumps(entry))
    with pytest.raises(Tuned):   # falls through to tuning (here: the stubbed library call)
        B.batched_tune(2, nmax=160, cache=str(path))


def test_tile_table_is_checked_before_any_call():
    H = torch.zeros(16, dtype=torch.complex128)
    L = torch.zeros(32, dtype=torch.complex128)
    for bad in ([0] * 3, [4] * B.LB_TILE_BUCKETS, [-1] * B.LB_TILE_BUCKETS):
        with pytest.raises(ValueError):
            B.steady_state_batched([4], 2, H, L, tiles=bad)
