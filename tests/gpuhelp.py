"""Helpers shared by the GPU parity tests (device transfer, layouts)."""
import numpy as np


def torch():
    import torch as _t
    return _t


def build_and_load():
    from paper_1108_5359_gb300 import build, _abi
    build.build()
    return _abi.load()


def to_dev_cm(a, dtype=None, ld=None):
    """Host array (rows x cols) -> column-major CUDA tensor, optional ld."""
    t = torch()
    a = np.asarray(a)
    rows, cols = a.shape
    dtype = dtype or (t.float64 if a.dtype == np.float64 else t.float32)
    ld = ld or rows
    buf = t.zeros((cols, ld), dtype=dtype, device="cuda")
    buf[:, :rows] = t.as_tensor(np.ascontiguousarray(a.T), dtype=dtype,
                                device="cuda")
    return buf.t()[:rows, :]


def to_host(t_):
    return t_.detach().cpu().numpy().astype(np.float64)


def idx_dev(v):
    t = torch()
    return t.as_tensor(np.asarray(v, dtype=np.int32), device="cuda")


def relerr(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)
