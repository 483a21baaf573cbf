"""The autotuner's host logic on CPU, with the GPU timing and device queries
replaced by stubs: the candidate list (trajectory vs checkpoints within the
memory budget), the rule that keeps the fixed schedule unless another one is
faster by more than the timing noise, the JSON cache (written once, read back
without timing, re-timed with force) and the cache key's N buckets."""
import pytest

torch = pytest.importorskip("torch")

from paper_1905_11071_gb300 import _lib, tune  # noqa: E402


@pytest.fixture
def stubbed(tmp_path, monkeypatch):
    """tune with a private cache file, a fake device and scripted timings."""
    monkeypatch.setenv("SLISTA_TUNE_CACHE", str(tmp_path / "cache.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "Fake GPU")
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda device=None: (1 << 40, 1 << 40))
    times = {}
    calls = []

    def fake_time(s, B, C, lam, alpha, prec, reps):
        calls.append((s.tile_rows, s.backward, s.ckpt_every))
        return times.get((s.tile_rows, s.backward, s.ckpt_every), 10.0)
    monkeypatch.setattr(tune, "_time", fake_time)
    return times, calls


def _problem(m=256, N=10000, T=40):
    return torch.zeros(m, m), torch.zeros(N, m), torch.full((T,), 0.1)


def test_candidates_cover_both_backward_modes_within_budget():
    _lib.load()
    T = 40
    c = tune.candidates(256, 10000, T, "bf16x3", 1 << 40)
    modes = {(s.tile_rows, s.backward) for s in c}
    assert (0, "traj") in modes and (0, "ckpt") in modes
    assert {s.tile_rows for s in c} == {0, 64, 96, 128}
    assert c[0].tile_rows == 0 and c[0].backward == "traj" and c[0].ckpt_every == T  # the fixed schedule first
    # FP32 has no trajectory backward; a tiny budget leaves nothing
    assert all(s.backward == "ckpt" for s in tune.candidates(256, 10000, T, "fp32", 1 << 40))
    assert tune.candidates(256, 10000, T, "bf16x3", 1024) == []


def test_fixed_schedule_kept_within_noise_and_replaced_beyond(stubbed):
    times, calls = stubbed
    B, C, alpha = _problem()
    # another schedule 1 % faster: within the noise, the fixed one stays
    times[(64, "traj", 40)] = 9.9
    best, tried = tune.tune(B, C, 0.1, alpha, prec="bf16x3", force=True)
    assert (best.tile_rows, best.backward) == (0, "traj")
    assert len(tried) == len(calls) > 1
    # 5 % faster: it replaces the fixed one
    times[(64, "traj", 40)] = 9.5
    best, _ = tune.tune(B, C, 0.1, alpha, prec="bf16x3", force=True)
    assert (best.tile_rows, best.backward, best.ms) == (64, "traj", 9.5)


def test_cache_is_written_read_back_and_bypassed_by_force(stubbed):
    times, calls = stubbed
    B, C, alpha = _problem()
    times[(96, "ckpt", 7)] = 5.0
    best, _ = tune.tune(B, C, 0.1, alpha, prec="bf16x3")
    assert (best.tile_rows, best.backward, best.ckpt_every) == (96, "ckpt", 7)
    n = len(calls)
    again, tried = tune.tune(B, C, 0.1, alpha, prec="bf16x3")  # from the cache: no timing
    assert len(calls) == n and tried == [again]
    assert (again.tile_rows, again.backward, again.ckpt_every) == (96, "ckpt", 7)
    assert tune.lookup(None, 256, 10000, 40, "bf16x3") == again
    tune.tune(B, C, 0.1, alpha, prec="bf16x3", force=True)
    assert len(calls) > n


def test_cache_key_buckets_batch_sizes(stubbed):
    k = tune.key(None, 256, 10000, 40, "bf16x3")
    assert k == "Fake_GPU|m256|N16384|T40|bf16x3"
    assert tune.key(None, 256, 9000, 40, "bf16x3") == k          # same power-of-two bucket
    assert tune.key(None, 256, 20000, 40, "bf16x3") != k
    assert tune.key(None, 256, 10000, 40, "bf16") != k
    assert tune.lookup(None, 256, 12345, 40, "bf16x3") is None     # nothing cached yet
