"""Small helpers shared by the tests (bit unpacking, brute-force search on
tiny inputs).  Test-side only."""
import numpy as np


def bits(hv):
    """uint64 words [..., W] -> bit array [..., 64*W] (bit d = word d//64, bit d%64)."""
    hv = np.ascontiguousarray(hv, dtype="<u8")
    b = np.unpackbits(hv.view(np.uint8), axis=-1, bitorder="little")
    return b


def pack(bitarr):
    b = np.ascontiguousarray(bitarr, dtype=np.uint8)
    return np.packbits(b, axis=-1, bitorder="little").view("<u8")


def hamming_matrix(a, b):
    """All-pairs Hamming distances of packed HVs by unpacked-bit comparison."""
    A, B = bits(a).astype(np.int32), bits(b).astype(np.int32)
    return (A[:, None, :] != B[None, :, :]).sum(-1)
