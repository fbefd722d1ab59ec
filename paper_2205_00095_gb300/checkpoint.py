"""State checkpoints: the conserved state with the problem description, the time and the step
count, written with ``torch.save`` and read back with ``torch.load(weights_only=True)`` (plain
containers and tensors only), so a run can stop and resume bit for bit.  Host side only: the
state is copied to the host on save and placed on the requested device on load.
"""
from __future__ import annotations

import math

import torch

FORMAT = 1


def save(path: str, spec: dict, U: torch.Tensor, t: float = 0.0, step: int = 0) -> None:
    """Write U (5, n_elem, n_node, float64) with its spec, time and step count to path."""
    if U.dtype != torch.float64 or U.dim() != 3 or U.shape[0] != 5:
        raise ValueError("U must be a float64 tensor of shape (5, n_elem, n_node)")
    if not math.isfinite(float(t)):
        raise ValueError("t must be finite")
    torch.save({"format": FORMAT, "spec": spec, "U": U.detach().to("cpu").contiguous(),
                "t": float(t), "step": int(step)}, path)


def load(path: str, device: str | torch.device | None = None) -> dict:
    """Read a checkpoint: {"spec", "U", "t", "step"}, U on `device` (default: the host)."""
    d = torch.load(path, map_location="cpu", weights_only=True)
    if not isinstance(d, dict) or d.get("format") != FORMAT:
        raise ValueError(f"{path}: not a checkpoint of format {FORMAT}")
    U = d["U"]
    if device is not None:
        U = U.to(device)
    return {"spec": d["spec"], "U": U, "t": d["t"], "step": d["step"]}
