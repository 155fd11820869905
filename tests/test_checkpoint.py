"""The outer loop's checkpoint file (host logic, CPU only): a round trip
keeps every array bit for bit, a file of another shape, storage type or
format is refused, and an interrupted write leaves the previous checkpoint
in place."""
import pytest

torch = pytest.importorskip("torch")

from paper_2607_11952_gb300 import api  # noqa: E402


def _state(n1=5, n2=3, ld=128, dtype="bf16", t=2, seed=0):
    g = torch.Generator().manual_seed(seed)
    kdt = torch.bfloat16 if dtype == "bf16" else torch.float32
    return {"n1": n1, "n2": n2, "ld": ld, "dtype": dtype, "t": t,
            "K": torch.rand(n1, ld, generator=g).to(kdt),
            "log_u": torch.randn(n1, generator=g), "log_v": torch.randn(n2, generator=g),
            "extra": {"warm": "learned"}}


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_round_trip_is_exact(tmp_path, dtype):
    s = _state(dtype=dtype)
    p = str(tmp_path / "ck.pt")
    api.write_checkpoint(p, s)
    ck = api.read_checkpoint(p, 5, 3, 128, dtype)
    assert ck["t"] == 2 and ck["extra"] == {"warm": "learned"}
    for k in ("K", "log_u", "log_v"):
        assert ck[k].dtype == s[k].dtype
        assert torch.equal(ck[k], s[k])


def test_mismatches_are_refused(tmp_path):
    p = str(tmp_path / "ck.pt")
    api.write_checkpoint(p, _state())
    with pytest.raises(ValueError):
        api.read_checkpoint(p, 6, 3, 128, "bf16")      # other n1
    with pytest.raises(ValueError):
        api.read_checkpoint(p, 5, 3, 128, "f32")       # other storage type
    bad = _state()
    bad["K"] = bad["K"][:, :64]
    api.write_checkpoint(p, bad)
    with pytest.raises(ValueError):
        api.read_checkpoint(p, 5, 3, 128, "bf16")      # arrays disagree with the header
    torch.save({"something": 1}, p)
    with pytest.raises(ValueError):
        api.read_checkpoint(p, 5, 3, 128, "bf16")      # not this library's format


def test_interrupted_write_keeps_previous(tmp_path, monkeypatch):
    p = str(tmp_path / "ck.pt")
    api.write_checkpoint(p, _state(t=1))
    real_save = torch.save

    def failing_save(obj, f, *a, **kw):
        real_save(obj, f, *a, **kw)
        raise OSError("disk full")                     # the write dies after the bytes went out

    monkeypatch.setattr(torch, "save", failing_save)
    with pytest.raises(OSError):
        api.write_checkpoint(p, _state(t=2, seed=1))
    monkeypatch.setattr(torch, "save", real_save)
    ck = api.read_checkpoint(p, 5, 3, 128, "bf16")
    assert ck["t"] == 1 and torch.equal(ck["K"], _state(t=1)["K"])
    assert sorted(x.name for x in tmp_path.iterdir()) == ["ck.pt"]   # no temporary left behind
