"""Save and resume a compiled tuning space: table images, their names and (optionally)
a fitted weight matrix in one file, so that a server or autotuner restarts without
compiling its IR again and without refitting.

File layout (little-endian): 8-byte magic b"PMCKPT01", u32 table count, u32 weight
rows, u32 weight columns, u32 reserved; per table a u32 name length, the UTF-8 name,
a u32 word count and the image words; the weights as float64 [rows][columns]; a
trailing u32 CRC-32 over every byte before it.  Loading checks the CRC and the
layout, then registers each image through pm_table_load, which checks its structure
again before anything reaches a device.
"""
import struct
import zlib
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import binding as B

MAGIC = b"PMCKPT01"


@dataclass
class Checkpoint:
    table_ids: List[int]          # ids in the context the file was loaded into
    names: List[str]
    weights: Optional[np.ndarray]  # float64 [models][K], or None


def save(path: str, ctx: B.Context, table_ids: Sequence[int], names: Optional[Sequence[str]] = None,
         weights: Optional[np.ndarray] = None) -> None:
    names = list(names) if names is not None else [""] * len(table_ids)
    if len(names) != len(table_ids):
        raise ValueError("one name per table")
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if w is not None and w.ndim != 2:
        raise ValueError("weights must be [models][K]")
    rows, cols = (0, 0) if w is None else w.shape
    out = [MAGIC, struct.pack("<4I", len(table_ids), rows, cols, 0)]
    for tid, name in zip(table_ids, names):
        nb = name.encode("utf-8")
        img = ctx.table_image(int(tid)).astype("<u4")
        out += [struct.pack("<I", len(nb)), nb, struct.pack("<I", img.size), img.tobytes()]
    if w is not None:
        out.append(w.astype("<f8").tobytes())
    body = b"".join(out)
    with open(path, "wb") as f:
        f.write(body + struct.pack("<I", zlib.crc32(body)))


def load(path: str, ctx: B.Context) -> Checkpoint:
    with open(path, "rb") as f:
        raw = f.read()
    if len(raw) < len(MAGIC) + 20 or raw[:len(MAGIC)] != MAGIC:
        raise ValueError(f"{path}: not a table checkpoint")
    body, (crc,) = raw[:-4], struct.unpack("<I", raw[-4:])
    if zlib.crc32(body) != crc:
        raise ValueError(f"{path}: checksum mismatch")
    o = len(MAGIC)
    n, rows, cols, _ = struct.unpack_from("<4I", body, o)
    o += 16

    def take(nbytes):
        nonlocal o
        if o + nbytes > len(body):
            raise ValueError(f"{path}: truncated")
        b = body[o:o + nbytes]
        o += nbytes
        return b

    ids, names = [], []
    for _ in range(n):
        (ln,) = struct.unpack("<I", take(4))
        names.append(take(ln).decode("utf-8"))
        (nw,) = struct.unpack("<I", take(4))
        ids.append(ctx.table_load(np.frombuffer(take(4 * nw), dtype="<u4").astype(np.uint32)))
    weights = None
    if rows:
        weights = np.frombuffer(take(8 * rows * cols), dtype="<f8").astype(np.float64).reshape(rows, cols)
    if o != len(body):
        raise ValueError(f"{path}: trailing bytes")
    return Checkpoint(ids, names, weights)
