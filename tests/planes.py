"""Conversions between the GPU library's bit-planes and per-realization state arrays
(0/1/2 per node, the encoding of Appendix A.1) used by the oracle.  Test helpers only."""
import numpy as np

SIR, SIS, IC, LT = 0, 1, 2, 3


def lane_bits(planes_p: np.ndarray, r: int) -> np.ndarray:
    """Bit r of every node from one plane [n][W] (u32)."""
    return ((planes_p[:, r >> 5].astype(np.uint64) >> np.uint64(r & 31)) & np.uint64(1)).astype(np.uint8)


def states_from_planes(model: int, planes: np.ndarray, lanes) -> np.ndarray:
    """planes: [P][n][W] u32 -> [len(lanes)][n] u8 states."""
    planes = planes.astype(np.uint32)
    out = np.zeros((len(lanes), planes.shape[1]), dtype=np.uint8)
    for i, r in enumerate(lanes):
        p0 = lane_bits(planes[0], r)
        if model == SIR:
            p1 = lane_bits(planes[1], r)
            out[i] = np.where(p0 == 1, 1, np.where(p1 == 1, 2, 0))
        elif model == SIS:
            out[i] = p0
        else:
            p1 = lane_bits(planes[1], r)
            out[i] = np.where(p1 == 1, 1, np.where(p0 == 1, 2, 0))
    return out


def planes_from_states(model: int, states: np.ndarray) -> np.ndarray:
    """[R][n] u8 states -> [P][n][W] u32 planes."""
    R, n = states.shape
    W = (R + 31) // 32
    P = 1 if model == SIS else 2
    planes = np.zeros((P, n, W), dtype=np.uint64)
    for r in range(R):
        s = states[r]
        if model == SIR:
            b0, b1 = (s == 1), (s == 2)
        elif model == SIS:
            b0, b1 = (s == 1), None
        else:
            b0, b1 = (s != 0), (s == 1)
        planes[0, :, r >> 5] |= b0.astype(np.uint64) << np.uint64(r & 31)
        if b1 is not None:
            planes[1, :, r >> 5] |= b1.astype(np.uint64) << np.uint64(r & 31)
    return planes.astype(np.uint32)
