"""Checkpoint files: a graph's saved state (DamfGraph.save / damf_save_state plus the exported
adjacency) as one little-endian file with a header, read back for DamfGraph.restore.

Layout (all integers little-endian):

    offset 0   8 bytes   magic "DAMFCKP1"
    offset 8   uint32    format version (1)
    offset 12  uint32    header length H (bytes of JSON)
    offset 16  uint32    CRC-32 of the header
    offset 20  uint32    zero
    offset 24  H bytes   header: UTF-8 JSON {"config": {damf_config fields}, "updates_since_fold",
                         "arrays": [{"name", "dtype", "shape", "offset", "nbytes", "crc32"}]}
    then every array's raw bytes (C order) at its 64-byte aligned offset

Arrays: Ub, Vb, Zb, r (n x d float32), PU, PV, PUi, PVi (d x d float32), sigma, s0 (d float32),
indptr (int32, n + 1) and indices (int32, indptr[n]). Reading checks the magic, the version,
the header's and every array's CRC-32, the bounds of every array in the file and the shapes
against n and d, and raises ValueError on any mismatch (a truncated or corrupted file never
reaches the device). Files are written to a temporary name and renamed into place.
"""

from __future__ import annotations

import json
import os
import struct
import zlib

import numpy as np

MAGIC = b"DAMFCKP1"
VERSION = 1
_PREFIX = struct.Struct("<8sIIII")
_ALIGN = 64
_STATE_NXD = ("Ub", "Vb", "Zb", "r")
_STATE_DXD = ("PU", "PV", "PUi", "PVi")
_STATE_D = ("sigma", "s0")
_DTYPES = {"<f4": np.dtype("<f4"), "<i4": np.dtype("<i4")}


def _host(x, dtype) -> np.ndarray:
    if hasattr(x, "detach"):        # a torch tensor (device or host)
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=dtype)


def _expected_shapes(n: int, d: int, nnz: int) -> dict:
    shapes = {k: (n, d) for k in _STATE_NXD}
    shapes.update({k: (d, d) for k in _STATE_DXD})
    shapes.update({k: (d,) for k in _STATE_D})
    shapes.update({"indptr": (n + 1,), "indices": (nnz,)})
    return shapes


def write_checkpoint(path: str, ck: dict) -> int:
    """Writes a checkpoint dict (from DamfGraph.save) to `path`; returns the bytes written."""
    from ._lib import Config
    cfg = ck["cfg"]
    conf = {name: getattr(cfg, name) for name, _ in Config._fields_}
    n, d = int(conf["n"]), int(conf["d"])
    arrays = {k: _host(ck["state"][k], "<f4") for k in _STATE_NXD + _STATE_DXD + _STATE_D}
    arrays["indptr"] = _host(ck["indptr"], "<i4")
    arrays["indices"] = _host(ck["indices"], "<i4")
    nnz = int(arrays["indptr"][-1]) if arrays["indptr"].size else -1
    want = _expected_shapes(n, d, nnz)
    for k, a in arrays.items():
        if a.shape != want[k]:
            raise ValueError("checkpoint array %s has shape %s, expected %s" % (k, a.shape, want[k]))
    # the header holds the arrays' offsets, which follow the header: lay out with room for
    # hlen bytes of header until the header fits in that room, then pad it to hlen
    crcs = {k: zlib.crc32(memoryview(a).cast("B")) for k, a in arrays.items()}
    hlen = 1024
    while True:
        off = -(-(_PREFIX.size + hlen) // _ALIGN) * _ALIGN
        meta = []
        for k, a in arrays.items():
            meta.append({"name": k, "dtype": a.dtype.str, "shape": list(a.shape), "offset": off,
                         "nbytes": int(a.nbytes), "crc32": crcs[k]})
            off = -(-(off + a.nbytes) // _ALIGN) * _ALIGN
        header = json.dumps({"config": conf, "updates_since_fold": int(ck["updates_since_fold"]), "arrays": meta},
                            sort_keys=True).encode()
        if len(header) <= hlen:
            header = header.ljust(hlen)
            break
        hlen = len(header) + 256
    tmp = "%s.tmp%d" % (path, os.getpid())
    with open(tmp, "wb") as f:
        f.write(_PREFIX.pack(MAGIC, VERSION, len(header), zlib.crc32(header), 0))
        f.write(header)
        for m in meta:
            f.write(b"\0" * (m["offset"] - f.tell()))
            f.write(memoryview(arrays[m["name"]]).cast("B"))
        total = f.tell()
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)
    return total


def read_checkpoint(path: str, device=None) -> dict:
    """Reads a checkpoint file into the dict DamfGraph.restore takes: the state as torch tensors
    (on `device`, default the host), the adjacency as numpy arrays, the config as a damf_config."""
    import torch
    from ._lib import Config
    with open(path, "rb") as f:
        blob = f.read()
    if len(blob) < _PREFIX.size:
        raise ValueError("checkpoint %s: truncated prefix" % path)
    magic, version, hlen, hcrc, _ = _PREFIX.unpack_from(blob, 0)
    if magic != MAGIC:
        raise ValueError("checkpoint %s: not a DAMF checkpoint" % path)
    if version != VERSION:
        raise ValueError("checkpoint %s: format version %d, expected %d" % (path, version, VERSION))
    header = blob[_PREFIX.size:_PREFIX.size + hlen]
    if len(header) != hlen or zlib.crc32(header) != hcrc:
        raise ValueError("checkpoint %s: header damaged" % path)
    try:
        head = json.loads(header.decode())
        conf = head["config"]
        cfg = Config(**{name: conf[name] for name, _ in Config._fields_})
        meta = {m["name"]: m for m in head["arrays"]}
        usf = int(head["updates_since_fold"])
    except (ValueError, KeyError, TypeError) as e:
        raise ValueError("checkpoint %s: header unreadable (%s)" % (path, e)) from None
    n, d = int(cfg.n), int(cfg.d)
    arrays = {}
    for k in _STATE_NXD + _STATE_DXD + _STATE_D + ("indptr", "indices"):
        m = meta.get(k)
        if m is None:
            raise ValueError("checkpoint %s: array %s missing" % (path, k))
        dt = _DTYPES.get(m["dtype"])
        off, nbytes, shape = int(m["offset"]), int(m["nbytes"]), tuple(int(s) for s in m["shape"])
        if dt is None or off < _PREFIX.size + hlen or off + nbytes > len(blob) or \
                nbytes != dt.itemsize * int(np.prod(shape, dtype=np.int64)):
            raise ValueError("checkpoint %s: array %s out of bounds or inconsistent" % (path, k))
        raw = memoryview(blob)[off:off + nbytes]
        if zlib.crc32(raw) != int(m["crc32"]):
            raise ValueError("checkpoint %s: array %s damaged (CRC-32 mismatch)" % (path, k))
        arrays[k] = np.frombuffer(raw, dtype=dt).reshape(shape).copy()   # owns its memory
    want = _expected_shapes(n, d, int(arrays["indptr"][-1]) if arrays["indptr"].size == n + 1 else -1)
    for k, a in arrays.items():
        if a.shape != want[k]:
            raise ValueError("checkpoint %s: array %s has shape %s, expected %s" % (path, k, a.shape, want[k]))
    state = {k: torch.from_numpy(arrays[k].astype(np.float32, copy=False))
             for k in _STATE_NXD + _STATE_DXD + _STATE_D}
    if device is not None:
        state = {k: v.to(device) for k, v in state.items()}
    return {"state": state, "updates_since_fold": usf, "indptr": arrays["indptr"].astype(np.int32),
            "indices": arrays["indices"].astype(np.int32), "cfg": cfg}
