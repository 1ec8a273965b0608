"""Training recipe for the learned coefficient model (all work runs in the library's kernels:
dataset generation from the exact fits, initialisation, normalisation, tensor-core training).

Default recipe: 2^22 samples uniform on the model domain, batch 16384, Adam with the learning
rate decaying geometrically from 1e-2 to 1e-5 over 64000 steps (250 passes over the set,
about 3 s on one GB300).
"""
from __future__ import annotations

from . import native

N_SAMPLES = 1 << 22
BATCH = 16384
STEPS = 64000
LR = (1e-2, 1e-5)


def train(seed: int = 20220329, n: int = N_SAMPLES, batch: int = BATCH, steps: int = STEPS,
          lr=LR, device="cuda"):
    """Returns (params [BL_MLP_PARAMS] CUDA float32, loss history [steps] CUDA float32)."""
    import torch
    inputs = torch.empty((n, 3), dtype=torch.float32, device=device)
    targets = torch.empty((n, 7), dtype=torch.float32, device=device)
    native.blacklight_mlp_dataset(n, seed, inputs, targets)
    params = torch.empty(native.MLP_PARAMS, dtype=torch.float32, device=device)
    native.blacklight_mlp_init(params, seed + 1)
    native.blacklight_mlp_normalise(inputs, targets, params)
    hist = torch.empty(max(steps, 1), dtype=torch.float32, device=device)
    native.blacklight_mlp_train(params, inputs, targets, batch, steps, lr[0], lr[1],
                                loss_history=hist)
    return params, hist[:steps]
