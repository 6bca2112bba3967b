"""Occupancy maps from binary images (the paper's maps are binary images of
the scene, Sec. 4.3.2 "Task2Task generalization" and Sec. 3.2.3).

read_map(path) returns a uint8 grid, grid[cy, cx], nonzero = occupied,
ready for ``Sim(params, [grid, ...], ...)``.  The image's top row is the
map's highest y (images are stored top-down, the simulator's y axis points
up); pass flip=False to keep the row order.  Dark pixels are obstacles:
a cell is occupied when its luminance is below `threshold` (0..255), or,
with invert=True, above it.  Formats: PNG (8-bit grey, grey + alpha, RGB,
RGBA, palette, and 1/2/4-bit grey or palette; no interlacing), binary or
ASCII PGM / PBM, and .npy arrays (nonzero = occupied, used as is).
"""

from __future__ import annotations

import struct
import zlib

import numpy as np


def _paeth(a, b, c):
    p = a + b - c
    pa, pb, pc = abs(p - a), abs(p - b), abs(p - c)
    if pa <= pb and pa <= pc:
        return a
    return b if pb <= pc else c


def _unfilter(raw: bytes, h: int, stride: int, bpp: int) -> np.ndarray:
    """Undo the five PNG scanline filters (None, Sub, Up, Average, Paeth)."""
    out = np.zeros((h, stride), np.uint8)
    prev = np.zeros(stride, np.int32)
    pos = 0
    for y in range(h):
        ft = raw[pos]
        line = np.frombuffer(raw, np.uint8, stride, pos + 1).astype(np.int32)
        pos += stride + 1
        cur = np.zeros(stride, np.int32)
        if ft == 0:
            cur[:] = line
        elif ft == 1:
            for x in range(stride):
                cur[x] = (line[x] + (cur[x - bpp] if x >= bpp else 0)) & 0xFF
        elif ft == 2:
            cur[:] = (line + prev) & 0xFF
        elif ft == 3:
            for x in range(stride):
                left = cur[x - bpp] if x >= bpp else 0
                cur[x] = (line[x] + ((left + prev[x]) >> 1)) & 0xFF
        elif ft == 4:
            for x in range(stride):
                left = cur[x - bpp] if x >= bpp else 0
                ul = prev[x - bpp] if x >= bpp else 0
                cur[x] = (line[x] + _paeth(left, prev[x], ul)) & 0xFF
        else:
            raise ValueError(f"bad PNG filter type {ft}")
        out[y] = cur
        prev = cur
    return out


def _read_png(data: bytes) -> np.ndarray:
    """Luminance (0..255, float) of a non-interlaced PNG."""
    if data[:8] != b"\x89PNG\r\n\x1a\n":
        raise ValueError("not a PNG file")
    pos, idat, palette = 8, [], None
    w = h = depth = ctype = interlace = None
    while pos < len(data):
        n, kind = struct.unpack(">I4s", data[pos:pos + 8])
        body = data[pos + 8:pos + 8 + n]
        pos += 12 + n
        if kind == b"IHDR":
            w, h, depth, ctype, _, _, interlace = struct.unpack(">IIBBBBB", body)
        elif kind == b"PLTE":
            palette = np.frombuffer(body, np.uint8).reshape(-1, 3).astype(np.float64)
        elif kind == b"IDAT":
            idat.append(body)
        elif kind == b"IEND":
            break
    if w is None or interlace:
        raise ValueError("unsupported PNG (missing header or interlaced)")
    channels = {0: 1, 2: 3, 3: 1, 4: 2, 6: 4}[ctype]
    if depth == 16 or (depth < 8 and ctype not in (0, 3)):
        raise ValueError(f"unsupported PNG bit depth {depth} for colour type {ctype}")
    bits = depth * channels
    stride = (w * bits + 7) // 8
    rows = _unfilter(zlib.decompress(b"".join(idat)), h, stride, max(1, bits // 8))
    if depth < 8:
        px = np.unpackbits(rows, axis=1)[:, : w * depth].reshape(h, w, depth)
        vals = (px * (1 << np.arange(depth - 1, -1, -1))).sum(axis=2)
        if ctype == 3:
            return palette[vals] @ np.array([0.299, 0.587, 0.114])
        return vals * (255.0 / ((1 << depth) - 1))
    px = rows[:, : w * channels].reshape(h, w, channels).astype(np.float64)
    if ctype == 3:
        return palette[px[..., 0].astype(np.int64)] @ np.array([0.299, 0.587, 0.114])
    if channels >= 3:
        return px[..., :3] @ np.array([0.299, 0.587, 0.114])
    return px[..., 0]


def _read_pnm(data: bytes) -> np.ndarray:
    """Luminance (0..255) of a PBM (P1 / P4) or PGM (P2 / P5) file."""
    magic = data[:2]
    toks, pos = [], 2
    need = 2 if magic in (b"P1", b"P4") else 3
    while len(toks) < need:
        while data[pos:pos + 1].isspace():
            pos += 1
        if data[pos:pos + 1] == b"#":
            while data[pos:pos + 1] not in (b"\n", b""):
                pos += 1
            continue
        start = pos
        while not data[pos:pos + 1].isspace():
            pos += 1
        toks.append(int(data[start:pos]))
    w, h = toks[0], toks[1]
    if magic == b"P4":
        pos += 1
        rows = np.frombuffer(data, np.uint8, h * ((w + 7) // 8), pos).reshape(h, -1)
        return (1 - np.unpackbits(rows, axis=1)[:, :w]) * 255.0  # 1 = black
    if magic == b"P5":
        maxv = toks[2]
        pos += 1
        dt = np.uint8 if maxv < 256 else np.dtype(">u2")
        return np.frombuffer(data, dt, w * h, pos).reshape(h, w).astype(np.float64) * (255.0 / maxv)
    vals = np.array(data[pos:].split(), dtype=np.int64)
    if magic == b"P1":
        return (1 - vals[: w * h].reshape(h, w)) * 255.0
    if magic == b"P2":
        return vals[: w * h].reshape(h, w) * (255.0 / toks[2])
    raise ValueError("not a PBM/PGM file")


def read_map(path: str, threshold: float = 128.0, invert: bool = False, flip: bool = True) -> np.ndarray:
    """Occupancy grid (uint8, 1 = occupied) of a binary map image."""
    if str(path).endswith(".npy"):
        return (np.load(path) != 0).astype(np.uint8)
    with open(path, "rb") as f:
        data = f.read()
    lum = _read_png(data) if data[:4] == b"\x89PNG" else _read_pnm(data)
    occ = lum > threshold if invert else lum < threshold
    if flip:
        occ = occ[::-1]
    return np.ascontiguousarray(occ.astype(np.uint8))
