"""Helpers shared by the GPU tests: run one operation through the C ABI (via
the ctypes binding) and bring the result back as bytes for comparison with
the oracle.  Unpacking uses numpy directly, independently of the binding."""
import os

import numpy as np
import torch

from paper_0712_0121_gb300 import morph as M

NCORES = os.cpu_count() or 1


def unpack_words(t: torch.Tensor, W: int) -> np.ndarray:
    raw = t.cpu().numpy().view(np.uint8).reshape(t.shape[0], -1)
    return np.unpackbits(raw, axis=1, bitorder="little")[:, :W]


def padding_bits_zero(t: torch.Tensor, W: int) -> bool:
    raw = t.cpu().numpy().view(np.uint8).reshape(t.shape[0], -1)
    bits = np.unpackbits(raw, axis=1, bitorder="little")
    return not bits[:, W:].any()


def packed_op(op, img, sw, sh, ox, oy, word_bits=64, dst_word_bits=None, stride_pad=0):
    """Packed path through the ABI; returns (result bytes, dst Packed)."""
    H, W = img.shape
    src = M.pack(img, word_bits, stride=(W + word_bits - 1) // word_bits + stride_pad)
    dwb = dst_word_bits or word_bits
    dst = M.Packed.empty(W, H, dwb, stride=(W + dwb - 1) // dwb + stride_pad)
    dst.words.fill_(-1)  # every output bit must be written
    M.morph_rect(op, dst, src, sw, sh, ox, oy)
    torch.cuda.synchronize()
    return unpack_words(dst.words, W), dst


def to_rle(img, word_bits=64):
    H, W = img.shape
    src = M.pack(img, word_bits)
    cap = max(1, H * ((W + 1) // 2))
    dst = M.Rle.empty(W, H, cap)
    M.rle_from_bitmap(dst, src)
    return dst


def rle_op(op, img, sw, sh, ox, oy, capacity=None):
    """RLE path: oracle-encoded input uploaded, op through the ABI, runs back."""
    import oracle
    H, W = img.shape
    rp, runs = oracle.rle_encode(img)
    src = M.Rle.from_numpy(rp, runs, W)
    cap = capacity if capacity is not None else max(1, H * ((W + 1) // 2))
    dst = M.Rle.empty(W, H, cap)
    M.morph_rect(op, dst, src, sw, sh, ox, oy)
    st = M.sync_status()
    return dst, st
