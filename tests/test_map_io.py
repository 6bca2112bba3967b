"""Binary-image map ingestion: grids written by an independent encoder in
this file (PNG through zlib with every scanline filter, PGM, PBM) read back
to the same occupancy, with the image's top row as the map's highest y."""

import struct
import zlib

import numpy as np
import pytest

from paper_2305_04180_gb300.map_io import read_map


def _png(path, pixels, ctype, depth=8, filt=0, palette=None):
    """Minimal PNG writer: one IDAT, every row with filter `filt` (the
    filtered bytes computed here from the definitions)."""
    h = pixels.shape[0]
    if depth < 8:
        rows = np.packbits(np.unpackbits(pixels.astype(np.uint8)[..., None], axis=2)[..., 8 - depth:].reshape(h, -1),
                           axis=1)
        bpp = 1
    else:
        rows = pixels.reshape(h, -1).astype(np.uint8)
        bpp = {0: 1, 2: 3, 3: 1, 4: 2, 6: 4}[ctype]
    raw = bytearray()
    prev = np.zeros(rows.shape[1], np.int32)
    for y in range(h):
        cur = rows[y].astype(np.int32)
        left = np.concatenate([np.zeros(bpp, np.int32), cur[:-bpp]])
        ul = np.concatenate([np.zeros(bpp, np.int32), prev[:-bpp]])
        if filt == 0:
            f = cur
        elif filt == 1:
            f = cur - left
        elif filt == 2:
            f = cur - prev
        elif filt == 3:
            f = cur - ((left + prev) >> 1)
        else:
            p = left + prev - ul
            pa, pb, pc = np.abs(p - left), np.abs(p - prev), np.abs(p - ul)
            pred = np.where((pa <= pb) & (pa <= pc), left, np.where(pb <= pc, prev, ul))
            f = cur - pred
        raw += bytes([filt]) + (f & 0xFF).astype(np.uint8).tobytes()
        prev = cur

    def chunk(kind, body):
        return struct.pack(">I", len(body)) + kind + body + struct.pack(">I", zlib.crc32(kind + body) & 0xFFFFFFFF)

    w = pixels.shape[1]
    out = b"\x89PNG\r\n\x1a\n" + chunk(b"IHDR", struct.pack(">IIBBBBB", w, h, depth, ctype, 0, 0, 0))
    if palette is not None:
        out += chunk(b"PLTE", np.asarray(palette, np.uint8).tobytes())
    out += chunk(b"IDAT", zlib.compress(bytes(raw))) + chunk(b"IEND", b"")
    path.write_bytes(out)


def _occupancy(seed, h=23, w=37):
    return (np.random.default_rng(seed).random((h, w)) < 0.3).astype(np.uint8)


@pytest.mark.parametrize("filt", [0, 1, 2, 3, 4])
def test_png_grey_every_filter(tmp_path, filt):
    occ = _occupancy(filt)
    img = np.where(occ, 0, 255)[::-1]  # dark = obstacle, top row = highest y
    _png(tmp_path / "m.png", img, 0, filt=filt)
    assert np.array_equal(read_map(str(tmp_path / "m.png")), occ)


def test_png_colour_alpha_palette_and_1bit(tmp_path):
    occ = _occupancy(7)
    img = np.where(occ, 0, 255)[::-1].astype(np.uint8)
    rgb = np.stack([img, img, img], axis=2)
    _png(tmp_path / "rgb.png", rgb, 2, filt=4)
    rgba = np.concatenate([rgb, np.full(img.shape + (1,), 255, np.uint8)], axis=2)
    _png(tmp_path / "rgba.png", rgba, 6, filt=1)
    ga = np.stack([img, np.full_like(img, 255)], axis=2)
    _png(tmp_path / "ga.png", ga, 4, filt=3)
    _png(tmp_path / "pal.png", (img > 0).astype(np.uint8), 3, palette=[[10, 10, 10], [250, 250, 250]], filt=2)
    _png(tmp_path / "bit.png", (img > 0).astype(np.uint8), 0, depth=1, filt=0)
    for name in ("rgb", "rgba", "ga", "pal", "bit"):
        assert np.array_equal(read_map(str(tmp_path / f"{name}.png")), occ), name


def test_pgm_pbm_npy_threshold_invert_flip(tmp_path):
    occ = _occupancy(9, 11, 13)
    img = np.where(occ, 20, 230).astype(np.uint8)[::-1]
    h, w = img.shape
    (tmp_path / "m.pgm").write_bytes(b"P5\n# comment\n%d %d\n255\n" % (w, h) + img.tobytes())
    (tmp_path / "a.pgm").write_bytes(b"P2\n%d %d\n255\n" % (w, h) + " ".join(map(str, img.ravel())).encode())
    bits = occ[::-1]  # PBM: 1 = black = occupied
    (tmp_path / "m.pbm").write_bytes(b"P4\n%d %d\n" % (w, h) + np.packbits(bits, axis=1).tobytes())
    (tmp_path / "a.pbm").write_bytes(b"P1\n%d %d\n" % (w, h) + " ".join(map(str, bits.ravel())).encode())
    np.save(tmp_path / "m.npy", occ)
    for name in ("m.pgm", "a.pgm", "m.pbm", "a.pbm", "m.npy"):
        assert np.array_equal(read_map(str(tmp_path / name)), occ), name
    assert np.array_equal(read_map(str(tmp_path / "m.pgm"), invert=True), 1 - occ)
    assert np.array_equal(read_map(str(tmp_path / "m.pgm"), flip=False), occ[::-1])
    assert np.array_equal(read_map(str(tmp_path / "m.pgm"), threshold=10), np.zeros_like(occ))
