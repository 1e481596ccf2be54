"""Host-side reading of the library's word layout (documented in include/mwmm.h)."""
import numpy as np


def unpack_words(buf: np.ndarray, words: int, nkb: int, rows_pad: int, kind: str, wpad: int = 0,
                 kmajor: bool = False) -> np.ndarray:
    """buf: uint8 bytes of one side's word region.  Returns [words][rows_pad][nkb*kb_elems]
    as float64: FP64 words ("fp64"), digits stored as bf16 ("int8") or as fp16
    ("f16", the 9-bit digits).  wpad > 0 or
    kmajor: the k-block-major layout with wpad zero words on each side (checked zero)."""
    if wpad or kmajor:
        wp = words + 2 * wpad
        a = np.asarray(buf[:nkb * wp * rows_pad * 128]).reshape(nkb, wp, rows_pad, 8, 16)
        assert not a[:, :wpad].any() and not a[:, wpad + words:].any(), "padding words must be zero"
        a = np.ascontiguousarray(a[:, wpad:wpad + words].transpose(1, 0, 2, 3, 4))
    else:
        n = words * nkb * rows_pad * 128
        a = np.asarray(buf[:n]).reshape(words, nkb, rows_pad, 8, 16)
    r = np.arange(rows_pad) & 7
    out = np.empty_like(a)
    for g in range(8):
        # logical granule g of row r sits at position g ^ (r & 7)
        out[:, :, :, g, :] = a[:, :, np.arange(rows_pad), g ^ r, :]
    if kind == "fp64":
        el = out.reshape(words, nkb, rows_pad, 128).view(np.float64)          # 16 per chunk
    elif kind == "f16":
        el = out.reshape(words, nkb, rows_pad, 128).view(np.float16).astype(np.float64)  # 64 fp16 per chunk
    else:
        u16 = out.reshape(words, nkb, rows_pad, 128).view(np.uint16)          # 64 bf16 per chunk
        el = (u16.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    kbe = el.shape[-1]
    return el.transpose(0, 2, 1, 3).reshape(words, rows_pad, nkb * kbe)
