"""Helpers for the learned decode proposal (see fgmm_mlp_* in include/fgmm.h).

The network's parameter vector theta (fp32, FGMM_MLP_PARAMS values) is laid
out as W1[10][64], b1[64], W2[64][64], b2[64], w3[64], b3. This module only
creates an initial theta; training, packing and inference run in the CUDA
library through codec.MlpTrainer / codec.mlp_pack / codec.decode_proposal.
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID = 10, 64
N_PARAMS = N_IN * N_HID + N_HID + N_HID * N_HID + N_HID + N_HID + 1


def init_theta(seed: int) -> np.ndarray:
    """Seeded uniform fan-in initialisation: weights ~ U(-a, a) with
    a = sqrt(3 / fan_in), biases 0."""
    rng = np.random.default_rng(seed)
    w1 = rng.uniform(-1, 1, (N_IN, N_HID)) * np.sqrt(3.0 / N_IN)
    w2 = rng.uniform(-1, 1, (N_HID, N_HID)) * np.sqrt(3.0 / N_HID)
    w3 = rng.uniform(-1, 1, N_HID) * np.sqrt(3.0 / N_HID)
    return np.concatenate([w1.ravel(), np.zeros(N_HID), w2.ravel(), np.zeros(N_HID), w3, [0.0]]).astype(np.float32)
