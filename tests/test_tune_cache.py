"""Host logic of the launch-shape autotuner's file cache (no GPU): a stored
choice is found again under the same GPU name, library build and workload
key, and not under another GPU name or workload."""
import synth
from paper_2604_24091_gb300 import tune


def test_file_cache_round_trip(tmp_path, monkeypatch):
    import torch
    path = str(tmp_path / "sub" / "tune.json")
    monkeypatch.setenv("AKMC_TUNE_CACHE", path)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "GPU-A")
    monkeypatch.setattr(tune, "_cache", {})
    descs = synth.config_batched_eam(4)
    key = tune.workload_key(descs)
    fkey = tune._file_key(key, "GPU-A")
    tune._store(tune.cache_path(), fkey, (16, 0))
    # a hit: no scratch batch is built (Batch would need a GPU)
    monkeypatch.setattr(tune, "Batch", None)
    assert tune.tune(descs, synth.default_model()) == (16, 0)
    # another GPU name or another workload is a different entry
    assert tune._file_key(key, "GPU-B") != fkey
    assert tune._file_key(tune.workload_key(synth.config_uneven(5)), "GPU-A") != fkey
    # an entry that is not one of the candidates is ignored
    tune._store(path, fkey, (3, 3))
    monkeypatch.setattr(tune, "_cache", {})
    hit = tune._load(path)[fkey]
    assert hit == [3, 3] and tuple(hit) not in set(tune.CANDIDATES)


def test_cache_disabled_by_empty_path(monkeypatch):
    monkeypatch.setenv("AKMC_TUNE_CACHE", "")
    assert tune.cache_path() is None
