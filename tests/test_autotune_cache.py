"""The autotuner's on-disk cache (host logic only, no GPU).

A result stored for one (grid shape and faces, periodicity, marker-count
bucket, device, compute capability, method, arithmetic, field, basis) key is
returned by a later tune() call without timing anything; other keys miss; the
file survives concurrent additions of different keys and a corrupt file reads
as empty; a tuning in which no candidate can be set up fails with a message
naming the candidates.
"""

import json

import numpy as np
import pytest

from paper_1805_01113_gb300 import autotune


@pytest.fixture
def fake_device(monkeypatch):
    monkeypatch.setattr(autotune, "_device", lambda: ("GB300-test", (10, 3)))
    monkeypatch.setattr(autotune, "_CACHE", {})


def _faces(n):
    return [np.linspace(-1.0, 1.0, n + 1)] * 3


class _Shape:
    """Stands in for a (3, M) marker tensor: tune() reads only its shape before a cache hit."""

    def __init__(self, M):
        self.shape = (3, M)


def test_round_trip_and_miss(tmp_path, fake_device):
    path = str(tmp_path / "tune.json")
    k = autotune._key(_faces(64), (True, True, True), 5000, "exact", "f32")
    assert autotune.disk_load(path, k) is None
    times = {(3, 3, 3): 0.5, (4, 4, 2): 0.4}
    autotune.disk_store(path, k, (4, 4, 2), times)
    assert autotune.disk_load(path, k) == ((4, 4, 2), times)
    other = autotune._key(_faces(64), (True, True, False), 5000, "exact", "f32")
    assert autotune.disk_load(path, other) is None
    autotune.disk_store(path, other, (3, 3, 3), {(3, 3, 3): 0.7})
    assert autotune.disk_load(path, k) == ((4, 4, 2), times)
    assert len(json.load(open(path))) == 2


def test_tune_uses_the_file_without_timing(tmp_path, monkeypatch, fake_device):
    path = str(tmp_path / "tune.json")
    faces, periodic, M = _faces(128), (True, True, True), 61440
    k = autotune._key(faces, periodic, M, "exact", "f32")
    autotune.disk_store(path, k, (4, 3, 3), {(4, 3, 3): 0.2, (3, 3, 3): 0.3})
    monkeypatch.setenv(autotune.CACHE_ENV, path)

    def no_context(*a, **kw):
        raise AssertionError("a cache hit must not create contexts")

    monkeypatch.setattr(autotune.api, "Context", no_context)
    best, times = autotune.tune(faces, periodic, _Shape(M), None, None, None)
    assert best == (4, 3, 3) and times[(3, 3, 3)] == 0.3
    # Same power-of-two bucket of marker counts: still a hit.
    assert autotune.tune(faces, periodic, _Shape(M + 1000), None, None, None)[0] == (4, 3, 3)


def test_key_separates_device_and_capability(monkeypatch):
    monkeypatch.setattr(autotune, "_device", lambda: ("GB300-test", (10, 3)))
    a = autotune._key(_faces(32), (True,) * 3, 100, "exact", "f32")
    monkeypatch.setattr(autotune, "_device", lambda: ("GB300-test", (10, 0)))
    b = autotune._key(_faces(32), (True,) * 3, 100, "exact", "f32")
    assert a != b


def test_corrupt_file_reads_as_empty(tmp_path, fake_device):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    k = autotune._key(_faces(16), (True,) * 3, 10, "fast", "bf16")
    assert autotune.disk_load(str(path), k) is None
    autotune.disk_store(str(path), k, (3, 3, 3), {(3, 3, 3): 1.0})
    assert autotune.disk_load(str(path), k)[0] == (3, 3, 3)


def test_uncached_path_times_every_candidate_and_stores(tmp_path, monkeypatch, fake_device):
    """The timing loop itself, with the library and CUDA events replaced by fakes:
    every candidate is timed, the fastest median wins and is written to the file."""
    path = str(tmp_path / "tune.json")
    monkeypatch.setenv(autotune.CACHE_ENV, path)
    cost = {(3, 3, 3): 3.0, (4, 3, 3): 2.0, (4, 4, 3): 2.5, (4, 4, 2): 1.5, (5, 3, 3): 4.0, (3, 3, 2): 1.75}
    made = []

    class FakeTransfer:
        def close(self):
            pass

    class FakeContext:
        def __init__(self, faces, periodic, real, field, brick_log2, basis=4):
            self.b = tuple(brick_log2)
            made.append(self.b)

        def transfer(self, M):
            return FakeTransfer()

        def build_transfer(self, *a):
            FakeEvent.clock += cost[self.b]

        def interpolate(self, *a):
            pass

        def spread(self, *a):
            pass

        def close(self):
            pass

    class FakeEvent:
        clock = 0.0

        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = FakeEvent.clock

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(autotune.api, "Context", FakeContext)
    monkeypatch.setattr(autotune.torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(autotune.torch.cuda, "synchronize", lambda: None)
    import torch
    x = torch.zeros((3, 100))
    u = torch.zeros((3, 4, 4, 4))
    best, times = autotune.tune(_faces(64), (True,) * 3, x, None, u, None)
    assert best == (4, 4, 2)
    assert sorted(made) == sorted(autotune.CANDIDATES)
    assert times == cost
    k = autotune._key(_faces(64), (True,) * 3, 100, "exact", "f32")
    assert autotune.disk_load(path, k) == ((4, 4, 2), cost)


def test_key_separates_stretched_from_uniform_faces(fake_device):
    n = 32
    uniform = _faces(n)
    xi = np.linspace(0.0, 1.0, n + 1)
    stretched = [uniform[0], uniform[1], np.tanh(1.5 * (2 * xi - 1)) / np.tanh(1.5)]
    a = autotune._key(uniform, (True, True, False), 1000, "exact", "f32")
    b = autotune._key(stretched, (True, True, False), 1000, "exact", "f32")
    assert a != b
    assert a == autotune._key([f.copy() for f in uniform], (True, True, False), 1000, "exact", "f32")


def test_key_separates_basis_and_arithmetic(fake_device):
    f = _faces(16)
    k4 = autotune._key(f, (True,) * 3, 10, "exact", "f32", "f32", 4)
    k10 = autotune._key(f, (True,) * 3, 10, "exact", "f32", "f32", 10)
    k64 = autotune._key(f, (True,) * 3, 10, "exact", "f64", "f64", 4)
    assert len({k4, k10, k64}) == 3


def test_no_candidate_gives_a_clear_error(monkeypatch, fake_device):
    monkeypatch.delenv(autotune.CACHE_ENV, raising=False)

    def refuse(*a, **kw):
        raise ValueError("tile too large")

    monkeypatch.setattr(autotune.api, "Context", refuse)
    with pytest.raises(RuntimeError, match=r"no candidate tile shape.*\(3, 3, 3\): tile too large"):
        import torch
        autotune.tune(_faces(8), (True,) * 3, torch.zeros((3, 100)), None, torch.zeros((3, 8, 8, 8)), None,
                      candidates=[(3, 3, 3)])
