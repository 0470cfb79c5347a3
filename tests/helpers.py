"""Conversions between numpy key arrays (the oracle's side) and torch CUDA tensors."""
import numpy as np

import oracle as O


def to_dev(a, device="cuda"):
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).to(device)
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).to(device)
    return torch.from_numpy(a).to(device)


def to_np(t, dtype):
    """Tensor -> numpy array of `dtype` (np.uint32 / np.uint64 / np.float32 / np.uint16)."""
    a = t.detach().cpu().numpy()
    return a.view(dtype)


def np_dtype(kt):
    return {O.KT_U32: np.uint32, O.KT_U64: np.uint64, O.KT_F32: np.float32}[kt]


def ordered_dtype(kt):
    return np.uint64 if kt == O.KT_U64 else np.uint32


def same_bits(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    if a.dtype == np.float32:
        a = a.view(np.uint32)
    if b.dtype == np.float32:
        b = b.view(np.uint32)
    return a.shape == b.shape and np.array_equal(a, b)
