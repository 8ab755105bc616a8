"""Host copies of device buffers that the library exposes by address (cr_get_device_state).

The checker reads the GPU's own iterate through these views so that the oracle can
evaluate its metrics at exactly that point.  Only marshalling: torch wraps the raw
address through the CUDA array interface and copies it to the host.
"""
import numpy as np


class _View:
    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(s) for s in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def to_host(ptr: int, shape, typestr: str) -> np.ndarray:
    import torch
    torch.cuda.synchronize()
    return torch.as_tensor(_View(ptr, shape, typestr), device="cuda").cpu().numpy().copy()


def theta_f64(st: dict, N: int, dtype: str = "f32", fp16_exponent: int = 0) -> np.ndarray:
    """theta^(1)_l of a handle (cr_get_device_state) as an N x N float64 array."""
    ld = st["ld"]
    if dtype == "f32":
        t = to_host(st["theta"], (N, ld), "<f4").astype(np.float64)
    elif dtype == "f64":
        t = to_host(st["theta"], (N, ld), "<f8")
    elif dtype == "bf16":
        raw = to_host(st["theta"], (N, ld), "<u2").astype(np.uint32) << 16
        t = raw.view(np.float32).astype(np.float64)
    elif dtype == "f16":
        t = to_host(st["theta"], (N, ld), "<f2").astype(np.float64) * 2.0 ** (-fp16_exponent)
    else:
        raise ValueError(dtype)
    return np.ascontiguousarray(t[:, :N])


def iterate_state(st: dict, N: int, n: int, dtype: str = "f32", fp16_exponent: int = 0) -> dict:
    """The handle's iterate: theta (N x N), mu (N), y (shifted, N), xi (N x n), all float64."""
    return {"theta": theta_f64(st, N, dtype, fp16_exponent),
            "mu": to_host(st["mu"], (N,), "<f8"),
            "y": to_host(st["y"], (N,), "<f8"),
            "xi": to_host(st["xi"], (N, n), "<f8"),
            "sigma": st["sigma"]}
