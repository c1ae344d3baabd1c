"""Host logic of the launch-shape autotuner on the CPU: the cache key names the GPU, the
precision, the Nb mix and the size class of the work; the cache file is replaced atomically
and survives a damaged file; a cached choice is returned without timing anything; the tuning
sample holds enough tiles to fill the GPU."""
import json

from paper_2511_21031_gb300 import autotune, workloads


def _insts():
    return workloads.batched_instances(n=5, seed=3, edge_lo=5, edge_hi=12, n_steps=4)


def test_cache_key_names_gpu_precision_nb_mix_and_size_class(monkeypatch):
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "GPU-X")
    insts = _insts()
    k = autotune.batch_key(insts, "mixed")
    nbs = sorted({w.n_bins for w in insts})
    cells = sum(w.n_cells for w in insts)
    assert k == f"GPU-X|batch|mixed|nb{nbs}|cells~1e{len(str(cells)) - 1}"
    assert autotune.batch_key(insts, "fp64") != k
    assert autotune.batch_key(insts[:1], "mixed") != k or len(nbs) == 1


def test_cache_round_trip_and_damaged_file(tmp_path):
    path = str(tmp_path / "cache.json")
    assert autotune._load(path) == {}
    autotune._save(path, {"a": {"block_warps": 1}})
    assert autotune._load(path) == {"a": {"block_warps": 1}}
    assert [p.name for p in tmp_path.iterdir()] == ["cache.json"]   # no temporary left behind
    open(path, "w").write("{not json")
    assert autotune._load(path) == {}


def test_cached_choice_is_returned_without_timing(monkeypatch, tmp_path):
    monkeypatch.setattr(autotune, "_gpu_name", lambda: "GPU-X")
    insts = _insts()
    path = str(tmp_path / "cache.json")
    choice = dict(block_warps=1, ctas_per_sm=32, bins_per_grab=1, ms=1.0)
    json.dump({autotune.batch_key(insts, "mixed"): choice}, open(path, "w"))

    def no_timing(*a, **k):
        raise AssertionError("a cached choice must not be re-timed")
    monkeypatch.setattr(autotune, "_time_events", no_timing)
    got = autotune.tune_batch(insts, precision="mixed", cache_path=path)
    assert got == dict(choice, cached=True)


def test_candidate_sets_are_within_the_library_ranges():
    for w, c, g in autotune.BATCH_CANDIDATES:
        assert 1 <= w <= 16 and 1 <= c <= 32 and 1 <= g <= 8
    assert len(set(autotune.BATCH_CANDIDATES)) == len(autotune.BATCH_CANDIDATES) == 28
    assert all(1 <= w <= 16 for w in autotune.SOLVER_CANDIDATES)


def test_tuning_sample_grows_until_it_holds_enough_tiles():
    wl = workloads.config_grid128(edge=32)
    slices = workloads.sliced_instances(wl, 64)                  # 512 cells = 16 tiles each
    pick = autotune.sample_instances(slices, 4, 200, seed=1)
    assert len(pick) == 13 and pick == sorted(set(pick))         # ceil(200 / 16) instances
    small = autotune.sample_instances(slices, 4, 10, seed=1)
    assert len(small) == 4 and set(small) <= set(pick)           # the count floor, same order
    assert len(autotune.sample_instances(slices, 4, 10 ** 9, seed=1)) == 64  # all of them
    big = _insts()
    assert len(autotune.sample_instances(big, 3, 0, seed=2)) == 3
