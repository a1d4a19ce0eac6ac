"""Test-side conversions between the library's stamp encoding and the oracle's distances.

The library stores, per cell, the stamp 1 + (slice mod 255) of the last slice that set it
(0 = unset); the oracle stores the paper's distance (slices since set, 65535 = never).
Comparisons use the canonical form: the distance when the cell is active in the window
(< k), else 255.
"""
import numpy as np

INF = 65535
HEADER_BYTES = 96  # size of the checkpoint header written by sse_export_state


def stamp(slice_index: int) -> int:
    return 1 + slice_index % 255


def canonical_from_stamps(stamps: np.ndarray, slice_index: int, k: int) -> np.ndarray:
    cs = stamp(slice_index)
    s = stamps.astype(np.int32)
    age = (cs - s) % 255
    out = np.where((s != 0) & (age < k), age, 255)
    return out.astype(np.uint8)


def stamps_from_distances(dist: np.ndarray, slice_index: int, k: int) -> np.ndarray:
    """Stamps that reproduce the oracle's active cells and ages at the given slice."""
    cs = stamp(slice_index)
    d = dist.astype(np.int64)
    s = (cs - 1 - d) % 255 + 1
    return np.where(d < k, s, 0).astype(np.uint8)


def state_blob(header: bytes, sre_stamps: np.ndarray, sle_stamps: np.ndarray, pitch: int) -> bytes:
    """A checkpoint for sse_import_state: an exported header followed by the stamp arrays
    (SLEA rows padded to the device pitch with unset cells)."""
    r2, length = sle_stamps.shape
    sle = np.zeros((r2, pitch), np.uint8)
    sle[:, :length] = sle_stamps
    return header[:HEADER_BYTES] + sre_stamps.astype(np.uint8).tobytes() + sle.tobytes()


def to_device(pairs: np.ndarray):
    import torch
    a = np.ascontiguousarray(pairs, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32)).cuda()
