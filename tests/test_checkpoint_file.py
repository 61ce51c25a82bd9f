"""Checkpoint files on the host: the state and adjacency a checkpoint holds come back bit for
bit, in the stated little-endian layout, and a damaged, truncated or foreign file is refused
before anything reaches the device (fault injection by corrupting inputs on the host)."""

import os
import struct

import numpy as np
import pytest
import torch

from paper_2306_08967_gb300._lib import Config
from paper_2306_08967_gb300.checkpoint import MAGIC, read_checkpoint, write_checkpoint


def _ck(n=37, d=16, seed=0):
    rng = np.random.default_rng(seed)
    deg = rng.integers(0, 6, size=n)
    indptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    indices = rng.integers(0, n, size=int(indptr[-1])).astype(np.int32)
    st = {k: torch.from_numpy(rng.standard_normal((n, d)).astype(np.float32)) for k in ("Ub", "Vb", "Zb", "r")}
    st.update({k: torch.from_numpy(rng.standard_normal((d, d)).astype(np.float32)) for k in ("PU", "PV", "PUi", "PVi")})
    st.update({k: torch.from_numpy(rng.random(d).astype(np.float32)) for k in ("sigma", "s0")})
    cfg = Config(n=n, n_capacity=n + 8, m_capacity=4096, d=d, directed=1, alpha=0.15, eps=1e-5, refold_every=256,
                 rsvd_oversample=10, rsvd_power_iters=4, max_push_rounds=1000, precision=1, threshold=1)
    return {"state": st, "updates_since_fold": 5, "indptr": indptr, "indices": indices, "cfg": cfg}


def test_round_trip_is_bit_exact(tmp_path):
    ck = _ck()
    path = str(tmp_path / "g.damf")
    size = write_checkpoint(path, ck)
    assert size == os.path.getsize(path)
    assert [p.name for p in tmp_path.iterdir()] == ["g.damf"]          # written under a temporary name
    back = read_checkpoint(path)
    for k, v in ck["state"].items():
        assert back["state"][k].dtype == torch.float32 and torch.equal(back["state"][k], v), k
    assert np.array_equal(back["indptr"], ck["indptr"]) and np.array_equal(back["indices"], ck["indices"])
    assert back["updates_since_fold"] == 5
    for name, _ in Config._fields_:
        assert getattr(back["cfg"], name) == getattr(ck["cfg"], name), name


def test_layout_is_little_endian_and_aligned(tmp_path):
    import json
    ck = _ck(n=10, d=16)
    path = str(tmp_path / "g.damf")
    write_checkpoint(path, ck)
    blob = open(path, "rb").read()
    magic, version, hlen, _, zero = struct.unpack_from("<8sIIII", blob, 0)
    assert magic == MAGIC and version == 1 and zero == 0
    head = json.loads(blob[24:24 + hlen])
    for m in head["arrays"]:
        assert m["offset"] % 64 == 0 and m["offset"] >= 24 + hlen
    ub = next(m for m in head["arrays"] if m["name"] == "Ub")
    assert ub["dtype"] == "<f4" and ub["shape"] == [10, 16]
    assert blob[ub["offset"]:ub["offset"] + ub["nbytes"]] == ck["state"]["Ub"].numpy().astype("<f4").tobytes()


@pytest.mark.parametrize("where", ["array", "header", "magic", "version", "truncate"])
def test_damaged_files_are_refused(tmp_path, where):
    import json
    ck = _ck()
    path = str(tmp_path / "g.damf")
    write_checkpoint(path, ck)
    blob = bytearray(open(path, "rb").read())
    hlen = struct.unpack_from("<I", blob, 12)[0]
    if where == "array":
        zb = next(m for m in json.loads(bytes(blob[24:24 + hlen]))["arrays"] if m["name"] == "Zb")
        blob[zb["offset"] + zb["nbytes"] // 2] ^= 0x10          # one flipped bit in Zb
    elif where == "header":
        blob[24 + hlen // 2] ^= 0x01
    elif where == "magic":
        blob[0:8] = b"NOTDAMF!"
    elif where == "version":
        struct.pack_into("<I", blob, 8, 2)
    else:
        blob = blob[: len(blob) - 100]
    open(path, "wb").write(bytes(blob))
    with pytest.raises(ValueError):
        read_checkpoint(path)


def test_inconsistent_shapes_are_refused(tmp_path):
    ck = _ck()
    ck["state"]["Ub"] = ck["state"]["Ub"][:-1]
    with pytest.raises(ValueError):
        write_checkpoint(str(tmp_path / "g.damf"), ck)
    ck = _ck()
    ck["indices"] = ck["indices"][:-1]                          # fewer entries than indptr says
    with pytest.raises(ValueError):
        write_checkpoint(str(tmp_path / "h.damf"), ck)
