"""Device-resident scenes and contexts for the library (marshalling only).

Moves a seeded synthetic scene (package `synth`) into torch CUDA tensors in the
SoA layout of the C ABI and runs the library's contact assembly on it.
"""
from __future__ import annotations

import torch

from . import binding


def scene_to_device(scene, device="cuda") -> dict:
    f = lambda a: torch.as_tensor(a, dtype=torch.float64).to(device).contiguous()
    return {
        "pos": f(scene.pos.T.copy()),
        "vel": f(scene.vel.T.copy()),
        "omega": f(scene.omega.T.copy()),
        "radius": f(scene.radius),
        "inv_mass": f(scene.inv_mass),
        "inv_inertia": f(scene.inv_inertia),
    }


def assemble(ctx: binding.Context, scene, slots: int = 3, device="cuda"):
    """Upload `scene` and build its contacts; returns (device scene dict, contacts view)."""
    dev = scene_to_device(scene, device)
    con = ctx.assemble(dev, scene.floor_z, scene.gravity, scene.dt, scene.delta, scene.mu, slots,
                       getattr(scene, "walls", ()))
    return dev, con


class _DeviceArray:
    """Minimal __cuda_array_interface__ wrapper around a raw device pointer."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


_TYPESTR = {torch.float64: "<f8", torch.int32: "<i4", torch.int64: "<i8"}


def view(con, name: str, device="cuda") -> torch.Tensor:
    """Copy a context-owned contact array (raw device pointer) into a new tensor."""
    Nc = con.Nc
    count = {"body_a": Nc, "body_b": Nc, "phi": Nc, "frame": 9 * Nc, "point": 3 * Nc, "arm_a": 3 * Nc,
             "arm_b": 3 * Nc, "key": Nc, "r": con.P, "plane": Nc}[name]
    dt = {"body_a": torch.int32, "body_b": torch.int32, "key": torch.int64, "plane": torch.int32}.get(name,
                                                                                                    torch.float64)
    if count == 0:
        return torch.empty(0, dtype=dt, device=device)
    arr = _DeviceArray(getattr(con, name), count, _TYPESTR[dt])
    return torch.as_tensor(arr, device=device).clone()
