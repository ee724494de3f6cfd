"""Helpers for the GPU tests: move inputs to the device, lay out tiles."""
import numpy as np
import torch


def dev(a) -> torch.Tensor:
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def locs_dev(locs) -> torch.Tensor:
    """(2, n) array -> device tensor holding x[0..n) then y[0..n)."""
    return dev(np.ascontiguousarray(locs).reshape(-1))


def tiles_from_list(tile_list) -> torch.Tensor:
    """Stack host tiles (lower-tile order) into one contiguous device buffer."""
    return dev(np.stack(tile_list)).contiguous()


def tiles_to_list(buf: torch.Tensor, T: int, b: int) -> list:
    arr = buf.detach().cpu().numpy().reshape(-1)[: T * (T + 1) // 2 * b * b]
    return list(arr.reshape(T * (T + 1) // 2, b, b))


def rel(a, b) -> float:
    return abs(a - b) / abs(b)
