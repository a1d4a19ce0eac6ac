"""Test-side conversions between the library's stamp encoding and the oracle's distances.

The library stores, per cell, the stamp 1 + (slice mod M) of the last slice that set it
(0 = unset), M = 255 for 8-bit and 65535 for 16-bit cells; the oracle stores the paper's
distance (slices since set, 65535 = never). Comparisons use the canonical form: the
distance when the cell is active in the window (< k), else INACTIVE.
"""
import numpy as np

INF = 65535
INACTIVE = 65535
HEADER_BYTES = 104  # size of the checkpoint header written by sse_export_state


def modulus(stamp_bits: int = 8) -> int:
    return (1 << stamp_bits) - 1


def stamp(slice_index: int, stamp_bits: int = 8) -> int:
    return 1 + slice_index % modulus(stamp_bits)


def canonical_from_stamps(stamps: np.ndarray, slice_index: int, k: int, stamp_bits: int = 8) -> np.ndarray:
    m = modulus(stamp_bits)
    cs = stamp(slice_index, stamp_bits)
    s = stamps.astype(np.int64)
    age = (cs - s) % m
    return np.where((s != 0) & (age < k), age, INACTIVE).astype(np.uint16)


def canonical_from_distances(dist: np.ndarray, k: int) -> np.ndarray:
    d = dist.astype(np.int64)
    return np.where(d < k, d, INACTIVE).astype(np.uint16)


def oracle_canonical(orc, k: int) -> tuple[np.ndarray, np.ndarray]:
    """The oracle's state in canonical form (from its raw 16-bit distances)."""
    sre, sle = orc.raw()
    return canonical_from_distances(sre, k), canonical_from_distances(sle, k)


def stamps_from_distances(dist: np.ndarray, slice_index: int, k: int, stamp_bits: int = 8) -> np.ndarray:
    """Stamps that reproduce the oracle's active cells and ages at the given slice."""
    m = modulus(stamp_bits)
    cs = stamp(slice_index, stamp_bits)
    d = dist.astype(np.int64)
    s = (cs - 1 - d) % m + 1
    return np.where(d < k, s, 0).astype(np.uint8 if stamp_bits == 8 else np.uint16)


def state_blob(header: bytes, sre_stamps: np.ndarray, sle_stamps: np.ndarray, pitch: int) -> bytes:
    """A checkpoint for sse_import_state: an exported header followed by the stamp arrays
    (SLEA rows padded to the device pitch with unset cells)."""
    r2, length = sle_stamps.shape
    sle = np.zeros((r2, pitch), sle_stamps.dtype)
    sle[:, :length] = sle_stamps
    return header[:HEADER_BYTES] + sre_stamps.astype(sle_stamps.dtype).tobytes() + sle.tobytes()


def to_device(pairs: np.ndarray):
    import torch
    a = np.ascontiguousarray(pairs, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).cuda()
