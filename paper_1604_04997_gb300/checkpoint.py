"""Save and resume a compiled tuning space: table images, their names, optionally a
fitted weight matrix, and named arrays (for a whole space: its variants, offsets and
points; see tuning.save_space) in one file, so that a server or autotuner restarts
without compiling its IR again and without refitting.

File layout (little-endian): 8-byte magic b"PMCKPT01", u32 table count, u32 weight
rows, u32 weight columns, u32 named-array count; per table a u32 name length, the
UTF-8 name, a u32 word count and the image words; the weights as float64
[rows][columns]; per named array a u32 name length, the name, a u32 dtype-string
length, the numpy dtype string (little-endian numeric types only), a u32 rank, u64
extents and the data; a trailing u32 CRC-32 over every byte before it.  Loading
checks the CRC and the layout, then registers each image through pm_table_load,
which checks its structure again before anything reaches a device.
"""
import struct
import zlib
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import binding as B

MAGIC = b"PMCKPT01"


_DTYPES = ("<i1", "<i2", "<i4", "<i8", "<u1", "<u2", "<u4", "<u8", "<f4", "<f8", "|i1", "|u1", "|b1")


@dataclass
class Checkpoint:
    table_ids: List[int]          # ids in the context the file was loaded into
    names: List[str]
    weights: Optional[np.ndarray]  # float64 [models][K], or None
    arrays: Dict[str, np.ndarray] = field(default_factory=dict)


def save(path: str, ctx: B.Context, table_ids: Sequence[int], names: Optional[Sequence[str]] = None,
         weights: Optional[np.ndarray] = None, arrays: Optional[Dict[str, np.ndarray]] = None) -> None:
    names = list(names) if names is not None else [""] * len(table_ids)
    if len(names) != len(table_ids):
        raise ValueError("one name per table")
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float64)
    if w is not None and w.ndim != 2:
        raise ValueError("weights must be [models][K]")
    rows, cols = (0, 0) if w is None else w.shape
    arrays = {} if arrays is None else arrays
    out = [MAGIC, struct.pack("<4I", len(table_ids), rows, cols, len(arrays))]
    for tid, name in zip(table_ids, names):
        nb = name.encode("utf-8")
        img = ctx.table_image(int(tid)).astype("<u4")
        out += [struct.pack("<I", len(nb)), nb, struct.pack("<I", img.size), img.tobytes()]
    if w is not None:
        out.append(w.astype("<f8").tobytes())
    for name, a in arrays.items():
        a = np.asarray(a)
        a = a if a.flags.c_contiguous else np.array(a, order="C")   # keeps rank 0 (ascontiguousarray would not)
        a = a.astype(a.dtype.newbyteorder("<")) if a.dtype.byteorder == ">" else a
        dt = a.dtype.str
        if dt not in _DTYPES:
            raise ValueError(f"array {name!r}: dtype {dt} not storable")
        nb, db = name.encode("utf-8"), dt.encode()
        out += [struct.pack("<I", len(nb)), nb, struct.pack("<I", len(db)), db, struct.pack("<I", a.ndim),
                struct.pack(f"<{a.ndim}Q", *a.shape), a.tobytes()]
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
    n, rows, cols, n_arr = struct.unpack_from("<4I", body, o)
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
    arrays = {}
    for _ in range(n_arr):
        (ln,) = struct.unpack("<I", take(4))
        name = take(ln).decode("utf-8")
        (ld,) = struct.unpack("<I", take(4))
        dt = take(ld).decode()
        if dt not in _DTYPES:
            raise ValueError(f"{path}: array {name!r} has dtype {dt}")
        (nd,) = struct.unpack("<I", take(4))
        if nd > 8:
            raise ValueError(f"{path}: array {name!r} has rank {nd}")
        shape = struct.unpack(f"<{nd}Q", take(8 * nd))
        count = int(np.prod(shape, dtype=np.uint64)) if nd else 1
        a = np.frombuffer(take(count * np.dtype(dt).itemsize), dtype=dt).reshape(shape)
        arrays[name] = a.astype(a.dtype.newbyteorder("="))
    if o != len(body):
        raise ValueError(f"{path}: trailing bytes")
    return Checkpoint(ids, names, weights, arrays)
