"""Element types of the data in the precision form (test infrastructure, FP64 oracle).

The data matrix may be held in TF32: FP32 storage whose values take part in the method rounded
to TF32 (1 sign, 8 exponent and 10 fraction bits), round to nearest with ties away from zero --
the reading of the rounding the paper leaves open, the one the tensor cores' explicit TF32
conversion performs.  The oracle applies the same rounding by its definition on the FP32 bit
pattern and then computes in FP64.
"""
import numpy as np


def round_tf32(x) -> np.ndarray:
    """FP32 values rounded to TF32 (nearest, ties away from zero), returned as float32.

    With the 13 low fraction bits dropped, adding half their range (0x1000) to the magnitude bits
    before truncating rounds to nearest and carries ties away from zero (the sign bit is separate).
    Non-finite values are returned unchanged."""
    f = np.ascontiguousarray(x, dtype=np.float32)
    b = f.view(np.uint32)
    finite = (b & np.uint32(0x7F800000)) != np.uint32(0x7F800000)
    r = np.where(finite, (b + np.uint32(0x1000)) & np.uint32(0xFFFFE000), b).astype(np.uint32)
    return r.view(np.float32).reshape(f.shape)
