"""GB300-native QTT-accelerated PDIP Newton solves for frictional contact.

The compute path is the CUDA library `libqttpdip.so` (C ABI in
include/qttpdip.h); `binding` marshals torch CUDA tensors into it and
`workload` prepares device-resident scenes.  Nothing here computes on the CPU.
"""
from . import binding  # noqa: F401

__all__ = ["binding"]
