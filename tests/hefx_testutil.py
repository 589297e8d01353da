"""Helpers shared by the GPU tests: device buffers via torch, results back as numpy."""
import numpy as np
import torch


def to_dev(arr: np.ndarray) -> torch.Tensor:
    a = np.ascontiguousarray(arr, dtype=np.uint32)
    return torch.from_numpy(a.view(np.int32).copy()).cuda()


def to_host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.cpu().numpy().view(np.uint32)


def empty_dev(shape) -> torch.Tensor:
    return torch.empty(shape, dtype=torch.int32, device="cuda")
